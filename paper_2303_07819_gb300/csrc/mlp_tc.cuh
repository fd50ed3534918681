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
// The backward pass's image of W_l^T (l = 1, 2, 3): 128 rows (the layer's
// inputs) by K = the layer's outputs, the output layer's 4 padded to 16.
__host__ __device__ inline int tc_timage_k(int layer) { return layer == 3 ? 16 : 128; }

// One layer of the closure network on the device: FP32 master weights and
// biases, Adam's moments, the batch's gradients (zero between batches), and
// the BF16 copies each engine reads.
struct LayerDev {
    int nin, nout, kin, nop;       // logical and padded sizes
    float *W, *b;                  // FP32 master [nout][nin], [nout]
    float *mW, *vW, *mb, *vb;      // Adam moments
    float *gW, *gb;                // gradients [nop][kin] (padded), [nout]
    __nv_bfloat16 *Wb, *Wt;        // BF16 copies [nop][kin] and [kin][nop] (mma.sync engine)
    __nv_bfloat16 *Wc;             // BF16 image of W for the tcgen05 kernels (tc_core_index layout, [rows][kin])
    __nv_bfloat16 *Wtc;            // BF16 image of W^T for the tcgen05 backward pass ([128][tk])
    int tk;                        // K of the W^T image (tc_timage_k)
};

struct AdamHyper {
    float lr, beta1, beta2, eps;
    const long long *tstep;        // Adam's step count (device), already advanced for this step
};

// Adam on entry i of layer L (weight i < nout * nin, row-major, else bias
// i - nout * nin), then the entry's BF16 copies in every layout; the
// gradient is read through L2 (other CTAs added to it atomically) and zeroed
// so that the next batch's sums start from zero.  c1, c2: the bias
// corrections 1 - beta^t.
__device__ inline void adam_entry(const LayerDev &L, int i, const AdamHyper &h, float c1, float c2)
{
    const int nw = L.nout * L.nin;
    if (i < nw) {
        const int o = i / L.nin, k = i % L.nin;
        const float g = __ldcg(&L.gW[o * L.kin + k]);
        L.gW[o * L.kin + k] = 0.0f;
        const float m = h.beta1 * L.mW[i] + (1.0f - h.beta1) * g;
        const float v = h.beta2 * L.vW[i] + (1.0f - h.beta2) * g * g;
        L.mW[i] = m;
        L.vW[i] = v;
        const float w = L.W[i] - h.lr * (m / c1) / (sqrtf(v / c2) + h.eps);
        L.W[i] = w;
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        L.Wb[o * L.kin + k] = wb;
        L.Wt[k * L.nop + o] = wb;
        L.Wc[tc_core_index(o, k, L.kin)] = wb;
        L.Wtc[tc_core_index(k, o, L.tk)] = wb;
    } else if (i < nw + L.nout) {
        const int o = i - nw;
        const float g = __ldcg(&L.gb[o]);
        L.gb[o] = 0.0f;
        const float m = h.beta1 * L.mb[o] + (1.0f - h.beta1) * g;
        const float v = h.beta2 * L.vb[o] + (1.0f - h.beta2) * g * g;
        L.mb[o] = m;
        L.vb[o] = v;
        L.b[o] -= h.lr * (m / c1) / (sqrtf(v / c2) + h.eps);
    }
}

struct TcArgs {
    const float *X;                  // [n][16] raw features (device)
    float *Y;                        // [n][4] tendencies in physical units (device)
    long long n;
    const __nv_bfloat16 *W[4];       // BF16 weight images (tc_core_index layout): 128x16, 128x128, 128x128, 16x128
    const float *b[4];               // biases: 128, 128, 128, 4
    const float *mu_x, *sd_x, *mu_y, *sd_y;   // z-scoring of the inputs and outputs
    int *err;                        // set to 1 if a wait on the tensor cores ran out
};

// One training batch, forward and backward through the hidden layers, per
// 128-sample tile (k_train_tile_tc).  The buffers have Bp rows (the batch
// rounded up to 8); rows B .. Bp - 1 are padding (zero inputs, zero dL/dy).
struct TrainArgs {
    const float *X, *Y;              // the batch: [B][16] raw features, [B][4] raw targets (device)
    int B, Bp;
    const __nv_bfloat16 *W[4];       // forward images, as TcArgs::W
    const __nv_bfloat16 *Wt[4];      // backward images of W_l^T for l = 1, 2, 3 (tc_timage_k); Wt[0] unused
    const float *b[4];
    const float *mu_x, *sd_x, *mu_y, *sd_y;
    __nv_bfloat16 *xt;               // out: [16][Bp] z-scored inputs, transposed
    __nv_bfloat16 *Ht[3];            // out: [128][Bp] hidden activations, transposed
    __nv_bfloat16 *dyt;              // out: rows 0-3 of [8][Bp], dL/dy transposed
    __nv_bfloat16 *dZt[3];           // out: [128][Bp] dL/dz of the hidden layers' pre-activations, transposed
    double *loss;                    // += the batch's mean squared error (z-scored outputs)
    long long *tick;                 // += 1 (Adam's step count) unless null
    int *err;                        // set to 1 if a wait on the tensor cores ran out
};

// Weight and bias gradients of the batch: for each job, gW[m][n] += sum_k
// A[m][k] B[n][k] over m < M, n < nin, and gb[m] += sum_k A[m][k]
// (k_wgrad_tc; A = dL/dz transposed, B = the layer's input transposed, both
// with K = Bp columns).
struct WgradJob {
    int M, nin, ldw;
    const __nv_bfloat16 *A, *B;
    float *gW, *gb;
};
struct WgradArgs {
    WgradJob job[4];
    int njob, K;
    int *err;
};

size_t mlp_tc_smem();
cudaError_t mlp_tc_prepare();
// a persistent grid of at most sm_count CTAs, 128 cells per tile
cudaError_t launch_mlp_forward_tc(const TcArgs &a, int sm_count, cudaStream_t st);

cudaError_t mlp_train_tc_prepare();
// one CTA per SM (210 KB of shared memory, all 512 tensor-memory columns), 128 samples per tile
cudaError_t launch_train_tile_tc(const TrainArgs &a, int sm_count, cudaStream_t st);
// the jobs' 64-column tiles times k slices of at least 64, about 2 CTAs per SM
cudaError_t launch_wgrad_tc(const WgradArgs &a, int sm_count, cudaStream_t st);

}  // namespace msd
