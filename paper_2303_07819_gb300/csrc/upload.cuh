// upload.cuh -- the caller's floes (FP64, the caller's order) into the cell
// layout on the device: the per-floe checks of ms_set_floes and the
// conversion to the stored state run as kernels over a raw device copy of
// the eight input arrays.
#pragma once
#include "common.cuh"

namespace msd {

// raw = device [8][n] doubles: x, y, theta, u, v, omega, r, h (caller's order)
struct UpGeom {
    long long n;
    int nx, ny;                 // cells (ny counts every stacked realization)
    double Lx, Ly, Lcx, Lcy;    // domain (all realizations) and cell sides
};

// cell_of[l] = the cell of caller floe l (x, y at raw[l], raw[n + l]: each
// coordinate wrapped into the periodic domain, then the half-open cell
// holding it); count[c] += the floes of cell c unless count is NULL
cudaError_t launch_cell_of(const double *raw, UpGeom g, int *cell_of, int *count, cudaStream_t st);

// The floes grouped by cell, a counting sort: given cell_of (n) and count
// (ncell, the floes per cell), off = the cells' first stored floe
// (exclusive scan, off[ncell] = n) and orig = caller indices grouped by
// cell, ascending within each cell.  cursor: ncell ints of scratch; tmp:
// sort_scan_ints(ncell + 1) ints of scratch.
long long sort_scan_ints(long long n);
cudaError_t sort_by_cell(const int *cell_of, const int *count, int *off, int *cursor, int *orig, int *tmp,
                         int ncell, long long n, cudaStream_t st);

// first[0] = smallest index with a non-finite value or r <= 0 or h <= 0,
// first[1] = smallest index (among the rest) whose cell is not cell_of[l];
// both stay ~0ull where there is none.  first must hold ~0ull on entry.
cudaError_t launch_check_floes(const double *raw, const int *cell_of, UpGeom g, unsigned long long *first,
                               cudaStream_t st);

// stored floe k = caller's floe orig[k] of cell cell_of[orig[k]]
cudaError_t launch_floes_to_cells32(const double *raw, const int *orig, const int *cell_of, UpGeom g,
                                    DevState32 s, cudaStream_t st);
cudaError_t launch_floes_to_cells64(const double *raw, const int *orig, const int *cell_of, UpGeom g,
                                    DevState64 s, cudaStream_t st);

}  // namespace msd
