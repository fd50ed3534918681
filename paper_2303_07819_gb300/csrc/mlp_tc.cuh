// mlp_tc.cuh -- closure network inference on the tcgen05 tensor cores.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace msd {

struct TcArgs {
    const float *X;                  // [n][16] raw features (device)
    float *Y;                        // [n][4] tendencies in physical units (device)
    long long n;
    const __nv_bfloat16 *W[4];       // BF16 weights [out_pad][in_pad] row-major: 128x16, 128x128, 128x128, 8x128
    const float *b[4];               // biases: 128, 128, 128, 4
    const float *mu_x, *sd_x, *mu_y, *sd_y;   // z-scoring of the inputs and outputs
    int nout_pad;                    // rows of W[3] (8)
    int *err;                        // set to 1 if a wait on the tensor cores ran out
};

size_t mlp_tc_smem();
cudaError_t mlp_tc_prepare();
// a persistent grid of at most sm_count CTAs, 128 cells per tile
cudaError_t launch_mlp_forward_tc(const TcArgs &a, int sm_count, cudaStream_t st);

}  // namespace msd
