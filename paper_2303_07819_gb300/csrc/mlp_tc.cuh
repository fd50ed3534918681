// mlp_tc.cuh -- closure network inference on the tcgen05 tensor cores.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace msd {

// Element index of weight (r, k) of an R x K layer in the kernel's
// shared-memory image: 8 x 8 "core matrices" (8 rows of 16 bytes), core
// matrix (i, j) at (i K/8 + j) 64 elements.  The weights are kept in this
// layout in global memory too, so a CTA stages them with bulk copies.
__host__ __device__ inline int tc_core_index(int r, int k, int K)
{
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
// rows of each layer's image: 128, 128, 128 and the output layer padded to 16
__host__ __device__ inline int tc_image_rows(int layer) { return layer == 3 ? 16 : 128; }

struct TcArgs {
    const float *X;                  // [n][16] raw features (device)
    float *Y;                        // [n][4] tendencies in physical units (device)
    long long n;
    const __nv_bfloat16 *W[4];       // BF16 weight images (tc_core_index layout): 128x16, 128x128, 128x128, 16x128
    const float *b[4];               // biases: 128, 128, 128, 4
    const float *mu_x, *sd_x, *mu_y, *sd_y;   // z-scoring of the inputs and outputs
    int *err;                        // set to 1 if a wait on the tensor cores ran out
};

size_t mlp_tc_smem();
cudaError_t mlp_tc_prepare();
// a persistent grid of at most sm_count CTAs, 128 cells per tile
cudaError_t launch_mlp_forward_tc(const TcArgs &a, int sm_count, cudaStream_t st);

}  // namespace msd
