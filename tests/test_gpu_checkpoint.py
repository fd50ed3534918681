"""Checkpoint and resume (ms_save / ms_load, the "save data" of Algorithm 1):
a run stopped, written to a file and loaded into a fresh model continues bit
for bit as the uninterrupted run, through coarse steps, gradual updates and
(FP32) the candidate lists kept across steps; the truth DEM likewise; files
of another model are refused."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def _same(a, b):
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.moments(), b.moments())
    ca, cb = a.coupling(), b.coupling()
    for k in ("q", "targets"):
        assert np.array_equal(ca[k], cb[k]), k


@pytest.mark.parametrize("precision, n1, n2", [(1, 130, 120), (0, 135, 100)])
def test_resume_equals_uninterrupted(ms, tmp_path, precision, n1, n2):
    """FP64 on the 4 x 4 square workload, stopped after 130 steps; FP32 on
    the batched workload's laws (16 x 16 cells), stopped after 135 steps,
    in the middle of a gradual-update period whose lists were built 4 steps
    before."""
    s = I.square_4x4() if precision == 1 else I.batched_128x128(seed=11, nx=16)
    p, fl, dt = s["params"], s["floes"], s["dt"]
    path = str(tmp_path / "run.ck")
    a = ms.Model(p, fl, precision)
    a.step(dt, n1 + n2)
    b = ms.Model(p, fl, precision)
    b.step(dt, n1)
    b.save(path)
    c = ms.Model(p, fl, precision)
    c.load_checkpoint(path)
    assert c.info()["steps"] == n1
    c.step(dt, n2)
    _same(a, c)
    for m in (a, b, c):
        m.close()


def test_truth_resume(ms, tmp_path):
    s = I.square_4x4()
    p, fl, dt = s["params"], s["floes"], s["dt"]
    path = str(tmp_path / "truth.ck")
    a = ms.Model(p, fl, ms.MS_FP64)
    a.truth_step(dt, 60)
    b = ms.Model(p, fl, ms.MS_FP64)
    b.truth_step(dt, 25)
    b.save(path)
    c = ms.Model(p, fl, ms.MS_FP64)
    c.load_checkpoint(path)
    c.truth_step(dt, 35)
    ta, tc = a.truth_floes(), c.truth_floes()
    for k in ta:
        assert np.array_equal(ta[k], tc[k]), k
    assert np.array_equal(a.truth_moments(), c.truth_moments())


def test_checkpoint_of_another_model_is_refused(ms, tmp_path):
    s = I.square_4x4()
    p, fl, dt = s["params"], s["floes"], s["dt"]
    path = str(tmp_path / "a.ck")
    a = ms.Model(p, fl, ms.MS_FP64)
    a.step(dt, 3)
    a.save(path)
    # other precision, fewer floes, a file that is no checkpoint, no file
    other = [ms.Model(p, fl, ms.MS_FP32),
             ms.Model(p, {k: v[:-1] for k, v in fl.items()}, ms.MS_FP64)]
    for m in other:
        with pytest.raises(ms.MsError) as e:
            m.load_checkpoint(path)
        assert e.value.code == -1
    bad = tmp_path / "bad.ck"
    bad.write_bytes(b"not a checkpoint at all")
    with pytest.raises(ms.MsError) as e:
        a.load_checkpoint(str(bad))
    assert e.value.code == -1
    with pytest.raises(ms.MsError) as e:
        a.load_checkpoint(str(tmp_path / "missing.ck"))
    assert e.value.code == -1


def _item_offsets(path):
    """(payload offset, bytes) of every item of a checkpoint file: an 8-byte
    tag, then per item an int64 byte count, the bytes and an 8-byte hash."""
    data = open(path, "rb").read()
    out, pos = [], 8
    while pos < len(data):
        nb = int(np.frombuffer(data[pos:pos + 8], dtype=np.int64)[0])
        out.append((pos + 8, nb))
        pos += 8 + nb + 8
    assert pos == len(data)
    return out


@pytest.mark.parametrize("which", ["list_head", "list_tail", "state"])
def test_corrupted_checkpoint_is_refused_and_changes_nothing(ms, tmp_path, which):
    """A checkpoint whose bytes were altered inside an item (list entries that
    would index past their cell, or a floe's state) is refused with
    MS_ERR_ARG before the model changes: the refused model then continues
    bit for bit as its untouched twin."""
    s = I.batched_128x128(seed=11, nx=16)
    p, fl, dt = s["params"], s["floes"], s["dt"]
    path = str(tmp_path / "c.ck")
    a = ms.Model(p, fl, ms.MS_FP32)
    a.step(dt, 23)
    a.save(path)
    items = _item_offsets(path)
    n = fl["x"].shape[0]
    # items: header, offsets, 8 state arrays, moments, window, q, targets,
    # control block, list heads, list tails, ...
    k = {"state": 5, "list_head": 15, "list_tail": 16}[which]
    off, nb = items[k]
    if which == "list_head":
        assert nb == 16 * n
    data = bytearray(open(path, "rb").read())
    for j in range(4):
        data[off + (nb // 3) + j] ^= 0xA5
    bad = str(tmp_path / "bad.ck")
    open(bad, "wb").write(bytes(data))
    b = ms.Model(p, fl, ms.MS_FP32)
    b.step(dt, 23)
    twin = ms.Model(p, fl, ms.MS_FP32)
    twin.step(dt, 23)
    with pytest.raises(ms.MsError) as e:
        b.load_checkpoint(bad)
    assert e.value.code == -1 and "checksum" in str(e.value)
    b.step(dt, 40)
    twin.step(dt, 40)
    _same(b, twin)
    for m in (a, b, twin):
        m.close()
