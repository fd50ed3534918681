// shard.cuh -- the device side of a grid split into tiles of cells, one per
// rank (Sec. 3.1's processor grid): what a rank sends and receives once per
// coarse interval.
#pragma once
#include <cuda_runtime.h>

namespace msd {

// a cell's coarse inputs: moment columns 1-5, then the five window sums
constexpr int SHARD_NCOL = 10;

// row k of send <- the coarse inputs of cells[k], k < ncells
cudaError_t launch_shard_pack(const double *mom, const double *win, int nc, const int *cells, int ncells,
                              double *send, cudaStream_t st);
// the coarse inputs of cells[t] <- row rows[t] of recv, t < nc (every cell)
cudaError_t launch_shard_scatter(double *mom, double *win, int nc, const int *cells, const long long *rows,
                                 const double *recv, cudaStream_t st);

}  // namespace msd
