"""Helpers shared by the parity tests: run the oracle and the CUDA path on the
same seeded inputs and compare per-cell moments field by field."""
import numpy as np

FIELDS = ["n", "M", "Mu", "Mv", "I", "Iw", "area", "Muu", "Mvv", "Fdx", "Fdy", "Td"]


def field_floors(ref: np.ndarray, params: dict, eps: float) -> np.ndarray:
    """Per-field floor of the relative error's denominator: eps times the
    field's natural scale (velocity 0.1 m/s, spin 1e-5 1/s), so fields that are
    near zero everywhere are compared against their scale, not against 0."""
    nM = np.linalg.norm(ref[:, 1])
    nI = np.linalg.norm(ref[:, 4])
    nA = np.linalg.norm(ref[:, 6])
    k = params.get("Cd", 0.0) * params.get("rho_o", 0.0)
    fl = np.array([1.0, nM, nM * 0.1, nM * 0.1, nI, nI * 1e-5, nA, nM * 1e-2, nM * 1e-2,
                   nA * k * 1e-2, nA * k * 1e-2, nI * k / max(params.get("rho_ice", 1.0), 1e-30) * 1e-10])
    return np.maximum(eps * fl, 1e-300)


def rel_errors(got: np.ndarray, ref: np.ndarray, params: dict, eps: float) -> np.ndarray:
    """||got_k - ref_k||_2 / max(||ref_k||_2, floor_k) for each moment column k
    (norm over cells)."""
    num = np.linalg.norm(got - ref, axis=0)
    den = np.maximum(np.linalg.norm(ref, axis=0), field_floors(ref, params, eps))
    return num / den


def report(errs: np.ndarray) -> str:
    return ", ".join(f"{n}={e:.2e}" for n, e in zip(FIELDS, errs))


def cell_errors(got: np.ndarray, ref: np.ndarray, params: dict, eps: float) -> np.ndarray:
    """Per moment column, the largest error of any single cell, over the
    column's rms across cells (floored as in rel_errors): a single cell that
    went wrong shows as an O(1) value however many cells agree."""
    n = ref.shape[0]
    rms = np.linalg.norm(ref, axis=0) / np.sqrt(max(n, 1))
    den = np.maximum(rms, field_floors(ref, params, eps) / np.sqrt(max(n, 1)))
    return np.max(np.abs(got - ref), axis=0) / den
