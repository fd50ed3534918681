// closure.cu -- the learned closure: a 16 -> 128 -> 128 -> 128 -> 4 tanh MLP
// that maps a cell's moments and forcing to its bulk drag tendencies, trained
// and evaluated with BF16 tensor-core products accumulated in FP32 (FP32
// master weights, Adam).
//
// Every product of the forward and backward pass is one call of a single
// tiled GEMM, C[m][n] = sum_k A[m][k] B[n][k], both operands BF16 with k
// contiguous, so the backward pass keeps each activation and each gradient in
// two layouts ([sample][unit] and [unit][sample]) written by the producing
// epilogue.  The weight gradients (sum over the batch) split the batch across
// blocks and add their partial products atomically.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "mlp_tc.cuh"
#include "../../include/msdem.h"

namespace msd {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NIN = 16, NH = 128, NOUT = 4;
constexpr int KIN = 16;          // input features padded to a multiple of 16
constexpr int NOP = 8;           // outputs padded to one n-tile
constexpr int BM = 64, BN = 64, BK = 32, SPAD = 8;

enum Epi { EPI_TANH = 0, EPI_LIN = 1, EPI_DZ = 2, EPI_F32 = 3 };

struct EpiArgs {
    const float *bias;     // EPI_TANH, EPI_LIN
    bf16 *out, *outT;      // EPI_TANH, EPI_DZ: [m][n] (ld ldo) and [n][m] (ld ldt)
    int ldo, ldt;
    const bf16 *h;         // EPI_DZ: the activation whose tanh' scales the product, [m][n] ld ldo
    float *bgrad;          // EPI_DZ: column sums (bias gradient), atomically
    float *f32;            // EPI_LIN, EPI_F32: FP32 result [m][n] ld ldf
    int ldf;
    int atomic;            // EPI_F32: add instead of store (split over k)
    int n_real;            // columns that exist (outputs beyond are padding)
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A B^T over a BM x BN tile per block (4 warps, 32 x 32 each), k-slice
// [kz * kchunk, (kz + 1) * kchunk) for blockIdx.z = kz.  lda, ldb and K are
// multiples of 8 (16-byte rows of BF16); out-of-range rows and k read as 0.
template <int EPI>
__global__ void __launch_bounds__(128)
k_gemm(int M, int N, int K, int kchunk, const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb,
       EpiArgs ea)
{
    __shared__ __align__(16) bf16 As[BM][BK + SPAD];
    __shared__ __align__(16) bf16 Bs[BN][BK + SPAD];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.0f;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // 64 rows x 4 chunks of 8 BF16 for each operand: 2 chunks per thread
        for (int c = threadIdx.x; c < BM * (BK / 8); c += 128) {
            const int r = c >> 2, kc = (c & 3) * 8;
            const int gk = k0 + kc;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M && gk < kend) va = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + gk);
            if (n0 + r < N && gk < kend) vb = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + gk);
            *reinterpret_cast<uint4 *>(&As[r][kc]) = va;
            *reinterpret_cast<uint4 *>(&Bs[r][kc]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = wm + 16 * i + g;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 8 + 2 * t]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = wn + 8 * j + g;
                bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t]);
                bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }

    // epilogue: element (m, n) of fragment value q: m = row + (q >= 2) * 8, n = col + (q & 1)
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float csum[2] = {0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int m = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (q & 1);
                float v = acc[i][j][q];
                const bool ok = m < M && n < N;
                if (EPI == EPI_TANH) {
                    if (ok) {
                        const float h = tanhf(v + ea.bias[n]);
                        const bf16 hb = __float2bfloat16_rn(h);
                        ea.out[(size_t)m * ea.ldo + n] = hb;
                        ea.outT[(size_t)n * ea.ldt + m] = hb;
                    }
                } else if (EPI == EPI_LIN) {
                    if (ok) ea.f32[(size_t)m * ea.ldf + n] = v + (n < ea.n_real ? ea.bias[n] : 0.0f);
                } else if (EPI == EPI_DZ) {
                    if (ok) {
                        const float h = __bfloat162float(ea.h[(size_t)m * ea.ldo + n]);
                        const float dz = v * (1.0f - h * h);
                        const bf16 db = __float2bfloat16_rn(dz);
                        ea.out[(size_t)m * ea.ldo + n] = db;
                        ea.outT[(size_t)n * ea.ldt + m] = db;
                        csum[q & 1] += dz;
                    }
                } else {
                    if (ok) {
                        float *p = ea.f32 + (size_t)m * ea.ldf + n;
                        if (ea.atomic) atomicAdd(p, v);
                        else *p = v;
                    }
                }
            }
            if (EPI == EPI_DZ) {
                // bias gradient: sum the column over the 8 row groups of the warp
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    float x = csum[s];
                    x += __shfl_xor_sync(0xffffffffu, x, 4);
                    x += __shfl_xor_sync(0xffffffffu, x, 8);
                    x += __shfl_xor_sync(0xffffffffu, x, 16);
                    const int n = n0 + wn + 8 * j + 2 * t + s;
                    if (g == 0 && n < N) atomicAdd(&ea.bgrad[n], x);
                }
            }
        }
}

// raw features -> z-scored BF16, [B][KIN] and [KIN][B] (padding columns 0)
__global__ void k_prep_input(const float *X, int B, int Bp, const float *mu, const float *sd, bf16 *xh, bf16 *xht)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Bp) return;
    for (int f = 0; f < KIN; f++) {
        float v = 0.0f;
        if (s < B && f < NIN) v = (X[(size_t)s * NIN + f] - mu[f]) / sd[f];
        const bf16 b = __float2bfloat16_rn(v);
        xh[(size_t)s * KIN + f] = b;
        xht[(size_t)f * Bp + s] = b;
    }
}

// z-scored residual of the outputs: loss sum, dL/dy in both layouts, output
// bias gradient (summed over the warp first: one atomic per warp and output)
__global__ void k_loss_grad(const float *yp, const float *Y, int B, int Bp, const float *mu, const float *sd,
                            bf16 *dy, bf16 *dyt, float *b4grad, double *loss)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    float gs[NOUT] = {};
    if (s < Bp) {
        for (int o = 0; o < NOP; o++) {
            float g = 0.0f;
            if (s < B && o < NOUT) {
                const float r = yp[(size_t)s * NOP + o] - (Y[(size_t)s * NOUT + o] - mu[o]) / sd[o];
                l += (double)r * r;
                g = 2.0f * r / (4.0f * (float)B);
                gs[o] = g;
            }
            const bf16 b = __float2bfloat16_rn(g);
            dy[(size_t)s * NOP + o] = b;
            dyt[(size_t)o * Bp + s] = b;
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
#pragma unroll
    for (int q = 0; q < NOUT; q++)
        for (int o = 16; o > 0; o >>= 1) gs[q] += __shfl_xor_sync(0xffffffffu, gs[q], o);
    if ((threadIdx.x & 31) == 0) {
        if (l != 0.0) atomicAdd(loss, l / (4.0 * B));
#pragma unroll
        for (int q = 0; q < NOUT; q++)
            if (gs[q] != 0.0f) atomicAdd(&b4grad[q], gs[q]);
    }
}

// z-scored outputs -> physical units
__global__ void k_denorm(const float *yp, int B, const float *mu, const float *sd, float *Y)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    for (int o = 0; o < NOUT; o++) Y[(size_t)s * NOUT + o] = mu[o] + sd[o] * yp[(size_t)s * NOP + o];
}

// Per-column mean and spread of a sample-major FP32 array [n][ncol], FP64
// sums: block b takes column b, each thread a strided share of the samples,
// then a fixed-order tree over the block (the same result on every run).
// out[b] = mean, out[ncol + b] = max(population sd, floor).
__global__ void __launch_bounds__(256) k_col_stats(const float *A, long long n, int ncol, double floor_sd,
                                                   double *out)
{
    __shared__ double red[256];
    const int col = blockIdx.x, t = threadIdx.x;
    auto block_sum = [&](double v) {
        red[t] = v;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (t < s) red[t] += red[t + s];
            __syncthreads();
        }
        const double r = red[0];
        __syncthreads();
        return r;
    };
    double s = 0.0;
    for (long long i = t; i < n; i += 256) s += (double)A[i * ncol + col];
    const double mean = block_sum(s) / (double)n;
    double q = 0.0;
    for (long long i = t; i < n; i += 256) {
        const double d = (double)A[i * ncol + col] - mean;
        q += d * d;
    }
    const double var = block_sum(q) / (double)n;
    if (t == 0) {
        out[col] = mean;
        out[ncol + col] = fmax(sqrt(var), floor_sd);
    }
}

// Adam on every layer in one launch.  Adam's step count lives on the device
// (so that a captured training epoch replays with the right bias
// corrections).
__global__ void k_tick(long long *t) { *t += 1; }

struct AdamAll {
    LayerDev L[4];
    int off[5];                // thread ranges: layer l takes [off[l], off[l+1])
    double *loss, *eloss;      // if eloss: the batch loss times B into eloss[*ep], the loss zeroed
    const int *ep;
    int B;
};

__global__ void k_adam(AdamAll A, AdamHyper h)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && A.eloss) {
        A.eloss[*A.ep] += *A.loss * A.B;
        *A.loss = 0.0;
    }
    if (i >= A.off[4]) return;
    int l = 0;
    while (i >= A.off[l + 1]) l++;
    const float tf = (float)*h.tstep;
    adam_entry(A.L[l], i - A.off[l], h, 1.0f - powf(h.beta1, tf), 1.0f - powf(h.beta2, tf));
}

// ---- the training loop's shuffle: a keyed permutation of [0, n), a
// four-round Feistel network on [0, 4^h) (4^h >= n), values past n walked
// on through the network until they fall below n (cycle walking; the walk
// returns to the domain because the start lies in it)

// integer mixer ("lowbias32", a published 32-bit hash)
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t feistel(uint32_t x, int h, uint4 k)
{
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = x >> h, R = x & mask;
    const uint32_t key[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const uint32_t nL = R;
        R = L ^ (mix32(R ^ key[r]) & mask);
        L = nL;
    }
    return (L << h) | R;
}

// Xs[i], Ys[i] = X[p(i)], Y[p(i)] for the epoch's permutation p
__global__ void k_gather_epoch(const float *X, const float *Y, long long n, int h, uint4 key, float *Xs, float *Ys)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = feistel((uint32_t)i, h, key);
    while (j >= (uint32_t)n) j = feistel(j, h, key);
#pragma unroll
    for (int f = 0; f < NIN; f++) Xs[i * NIN + f] = X[(long long)j * NIN + f];
#pragma unroll
    for (int o = 0; o < NOUT; o++) Ys[i * NOUT + o] = Y[(long long)j * NOUT + o];
}

__global__ void k_set_epoch(int *ep, int v) { *ep = v; }

// the batch's mean loss times its size into the current epoch's sum

__global__ void k_cast_layer(LayerDev L)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nop * L.kin) return;
    const int o = i / L.kin, k = i % L.kin;
    const float w = (o < L.nout && k < L.nin) ? L.W[o * L.nin + k] : 0.0f;
    const bf16 wb = __float2bfloat16_rn(w);
    L.Wb[i] = wb;
    L.Wt[k * L.nop + o] = wb;
    L.Wc[tc_core_index(o, k, L.kin)] = wb;
    if (o < L.tk) L.Wtc[tc_core_index(k, o, L.tk)] = wb;
}

}  // namespace

}  // namespace msd

using namespace msd;

struct ms_mlp {
    int max_batch = 0, bp = 0;
    LayerDev L[4];
    float *mu_x = nullptr, *sd_x = nullptr, *mu_y = nullptr, *sd_y = nullptr;
    float *X = nullptr, *Y = nullptr, *yp = nullptr, *yout = nullptr;
    bf16 *xh = nullptr, *xht = nullptr, *H[3] = {}, *Ht[3] = {}, *dZ[3] = {}, *dZt[3] = {}, *dy = nullptr,
         *dyt = nullptr;
    double *loss = nullptr;
    long long *d_t = nullptr;  // Adam steps (device)
    double *d_eloss = nullptr; // per-epoch loss sums of ms_mlp_train (device)
    int *d_ep = nullptr;       // the epoch being trained (device)
    int engine = 1;            // 1: tcgen05 (fused inference kernel, training GEMMs), 0: mma.sync tiles
    int sm_count = 0;
    int *tc_err = nullptr;     // set by the tcgen05 kernel if a wait ran out
    cudaStream_t st = nullptr;
    std::vector<void *> allocs;
    std::vector<float> hnorm;
};

namespace msd {

static const int LIN[4] = {NIN, NH, NH, NH}, LOUT[4] = {NH, NH, NH, NOUT};
static const int LKIN[4] = {KIN, NH, NH, NH}, LNOP[4] = {NH, NH, NH, NOP};

template <class T>
static cudaError_t mal(ms_mlp *m, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return cudaMemsetAsync(q, 0, sizeof(T) * (n ? n : 1), m->st);
}

// C = A B^T with epilogue epi on the MLP's stream (the mma.sync tiles)
static cudaError_t gemm(const ms_mlp *m, int epi, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb,
                        const EpiArgs &ea, int ksplit = 1)
{
    cudaStream_t st = m->st;
    const int kchunk = ((K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, (K + kchunk - 1) / kchunk);
    switch (epi) {
    case EPI_TANH: k_gemm<EPI_TANH><<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, ea); break;
    case EPI_LIN: k_gemm<EPI_LIN><<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, ea); break;
    case EPI_DZ: k_gemm<EPI_DZ><<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, ea); break;
    default: k_gemm<EPI_F32><<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, ea); break;
    }
    return cudaGetLastError();
}

// forward pass of a batch already z-scored in m->xh (Bp rows): m->yp = z-scored outputs
static cudaError_t forward(ms_mlp *m, int Bp)
{
    cudaError_t e;
    const bf16 *in = m->xh;
    int ldin = KIN;
    for (int l = 0; l < 3; l++) {
        EpiArgs ea{};
        ea.bias = m->L[l].b;
        ea.out = m->H[l];
        ea.outT = m->Ht[l];
        ea.ldo = NH;
        ea.ldt = Bp;
        if ((e = gemm(m, EPI_TANH, Bp, NH, LKIN[l], in, ldin, m->L[l].Wb, LKIN[l], ea)) != cudaSuccess) return e;
        in = m->H[l];
        ldin = NH;
    }
    EpiArgs ea{};
    ea.bias = m->L[3].b;
    ea.f32 = m->yp;
    ea.ldf = NOP;
    ea.n_real = NOUT;
    return gemm(m, EPI_LIN, Bp, NOP, NH, in, NH, m->L[3].Wb, NH, ea);
}

// gradients of the batch loss (z-scored units) added to the layers' gW, gb (zero
// at entry: Adam zeroes them once read) and the loss added to m->loss
static cudaError_t backward(ms_mlp *m, int B, int Bp)
{
    cudaError_t e;
    k_loss_grad<<<(Bp + 255) / 256, 256, 0, m->st>>>(m->yp, m->Y, B, Bp, m->mu_y, m->sd_y, m->dy, m->dyt, m->L[3].gb,
                                                     m->loss);
    const int ks = Bp >= 4096 ? 32 : (Bp >= 512 ? 8 : 1);
    // output layer: gW4 = dy^T H3, then the gradient through it
    const bf16 *dz = m->dy, *dzt = m->dyt;
    int ldz = NOP;
    for (int l = 3; l >= 0; l--) {
        const bf16 *xt = l > 0 ? m->Ht[l - 1] : m->xht;
        EpiArgs eg{};
        eg.f32 = m->L[l].gW;
        eg.ldf = LKIN[l];
        eg.atomic = ks > 1;
        if ((e = gemm(m, EPI_F32, LOUT[l], LKIN[l], Bp, dzt, Bp, xt, Bp, eg, ks)) != cudaSuccess) return e;
        if (l == 0) break;
        // dH_{l} = dz W_l -> dZ_{l-1} = dH (1 - h^2), plus its bias gradient
        EpiArgs ed{};
        ed.h = m->H[l - 1];
        ed.out = m->dZ[l - 1];
        ed.outT = m->dZt[l - 1];
        ed.ldo = NH;
        ed.ldt = Bp;
        ed.bgrad = m->L[l - 1].gb;
        if ((e = gemm(m, EPI_DZ, Bp, NH, LNOP[l], dz, ldz, m->L[l].Wt, LNOP[l], ed)) != cudaSuccess) return e;
        dz = m->dZ[l - 1];
        dzt = m->dZt[l - 1];
        ldz = NH;
    }
    return cudaGetLastError();
}

static int pad8(long long n) { return (int)((n + 7) / 8 * 8); }

}  // namespace msd

// ----------------------------------------------------------------- C-ABI
static int ms_closure_fail(int code, const char *msg) { return msd::set_error(code, msg); }

extern "C" {

static int ck(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MS_OK;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s failed: %s", what, cudaGetErrorString(e));
    return ms_closure_fail(MS_ERR_CUDA, buf);
}
#define CKC(x) do { int rc_ = ck((x), #x); if (rc_) return rc_; } while (0)

int ms_mlp_create(ms_mlp **out, const float *params, const float *norm, int32_t max_batch)
{
    if (!out || !params || !norm) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 22)) return ms_closure_fail(MS_ERR_ARG, "max_batch must be in [1, 2^22]");
    for (int i = 0; i < 2 * NIN + 2 * NOUT; i++)
        if (!std::isfinite(norm[i]) || (((i >= NIN && i < 2 * NIN) || i >= 2 * NIN + NOUT) && !(norm[i] > 0.0f)))
            return ms_closure_fail(MS_ERR_ARG, "normalisation needs finite means and positive spreads");
    ms_mlp *m = new ms_mlp();
    m->max_batch = max_batch;
    m->bp = pad8(max_batch);
    m->hnorm.assign(norm, norm + 2 * NIN + 2 * NOUT);
    int rc = MS_OK;
    auto fail_free = [&](int r) { ms_mlp_free(m); return r; };
    if ((rc = ck(cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking), "stream"))) return fail_free(rc);
    const int Bp = m->bp;
    size_t off = 0;
    for (int l = 0; l < 4; l++) {
        LayerDev &L = m->L[l];
        L.nin = LIN[l]; L.nout = LOUT[l]; L.kin = LKIN[l]; L.nop = LNOP[l]; L.tk = tc_timage_k(l);
        const size_t nw = (size_t)L.nout * L.nin;
        cudaError_t e;
        if ((e = mal(m, &L.W, nw)) || (e = mal(m, &L.b, L.nout)) || (e = mal(m, &L.mW, nw)) ||
            (e = mal(m, &L.vW, nw)) || (e = mal(m, &L.mb, L.nout)) || (e = mal(m, &L.vb, L.nout)) ||
            (e = mal(m, &L.gW, (size_t)L.nop * L.kin)) || (e = mal(m, &L.gb, L.nout)) ||
            (e = mal(m, &L.Wb, (size_t)L.nop * L.kin)) || (e = mal(m, &L.Wt, (size_t)L.nop * L.kin)) ||
            (e = mal(m, &L.Wc, (size_t)tc_image_rows(l) * L.kin)) || (e = mal(m, &L.Wtc, (size_t)NH * L.tk)))
            return fail_free(ck(e, "cudaMalloc"));
        if ((rc = ck(cudaMemcpyAsync(L.W, params + off, sizeof(float) * nw, cudaMemcpyHostToDevice, m->st), "copy")))
            return fail_free(rc);
        off += nw;
        if ((rc = ck(cudaMemcpyAsync(L.b, params + off, sizeof(float) * L.nout, cudaMemcpyHostToDevice, m->st), "copy")))
            return fail_free(rc);
        off += L.nout;
        k_cast_layer<<<(L.nop * L.kin + 255) / 256, 256, 0, m->st>>>(L);
    }
    cudaError_t e;
    if ((e = mal(m, &m->mu_x, NIN)) || (e = mal(m, &m->sd_x, NIN)) || (e = mal(m, &m->mu_y, NOUT)) ||
        (e = mal(m, &m->sd_y, NOUT)) || (e = mal(m, &m->X, (size_t)Bp * NIN)) || (e = mal(m, &m->Y, (size_t)Bp * NOUT)) ||
        (e = mal(m, &m->yp, (size_t)Bp * NOP)) || (e = mal(m, &m->yout, (size_t)Bp * NOUT)) ||
        (e = mal(m, &m->xh, (size_t)Bp * KIN)) || (e = mal(m, &m->xht, (size_t)Bp * KIN)) ||
        (e = mal(m, &m->dy, (size_t)Bp * NOP)) || (e = mal(m, &m->dyt, (size_t)Bp * NOP)) || (e = mal(m, &m->loss, 1)) ||
        (e = mal(m, &m->tc_err, 1)) || (e = mal(m, &m->d_t, 1)) || (e = mal(m, &m->d_ep, 1)))
        return fail_free(ck(e, "cudaMalloc"));
    {
        int dev = 0;
        if ((rc = ck(cudaGetDevice(&dev), "device")) ||
            (rc = ck(cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev), "attribute")) ||
            (rc = ck(mlp_tc_prepare(), "tcgen05 kernel attribute")) ||
            (rc = ck(mlp_train_tc_prepare(), "tcgen05 kernel attribute")))
            return fail_free(rc);
    }
    for (int l = 0; l < 3; l++)
        if ((e = mal(m, &m->H[l], (size_t)Bp * NH)) || (e = mal(m, &m->Ht[l], (size_t)Bp * NH)) ||
            (e = mal(m, &m->dZ[l], (size_t)Bp * NH)) || (e = mal(m, &m->dZt[l], (size_t)Bp * NH)))
            return fail_free(ck(e, "cudaMalloc"));
    const float *nz = m->hnorm.data();
    if ((rc = ck(cudaMemcpyAsync(m->mu_x, nz, 4 * NIN, cudaMemcpyHostToDevice, m->st), "copy")) ||
        (rc = ck(cudaMemcpyAsync(m->sd_x, nz + NIN, 4 * NIN, cudaMemcpyHostToDevice, m->st), "copy")) ||
        (rc = ck(cudaMemcpyAsync(m->mu_y, nz + 2 * NIN, 4 * NOUT, cudaMemcpyHostToDevice, m->st), "copy")) ||
        (rc = ck(cudaMemcpyAsync(m->sd_y, nz + 2 * NIN + NOUT, 4 * NOUT, cudaMemcpyHostToDevice, m->st), "copy")) ||
        (rc = ck(cudaStreamSynchronize(m->st), "sync")))
        return fail_free(rc);
    *out = m;
    return MS_OK;
}

int ms_mlp_fit_norm(const float *X, const float *Y, int64_t n, float *norm)
{
    if (!X || !Y || !norm) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (n < 1 || n > (int64_t(1) << 31)) return ms_closure_fail(MS_ERR_ARG, "n must be in [1, 2^31]");
    cudaStream_t st = nullptr;
    float *Xd = nullptr, *Yd = nullptr;
    double *sd = nullptr;
    int rc = ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    if (rc == MS_OK) rc = ck(cudaMalloc(&Xd, sizeof(float) * (size_t)n * NIN), "cudaMalloc");
    if (rc == MS_OK) rc = ck(cudaMalloc(&Yd, sizeof(float) * (size_t)n * NOUT), "cudaMalloc");
    if (rc == MS_OK) rc = ck(cudaMalloc(&sd, sizeof(double) * 2 * (NIN + NOUT)), "cudaMalloc");
    if (rc == MS_OK)
        rc = ck(cudaMemcpyAsync(Xd, X, sizeof(float) * (size_t)n * NIN, cudaMemcpyHostToDevice, st), "copy");
    if (rc == MS_OK)
        rc = ck(cudaMemcpyAsync(Yd, Y, sizeof(float) * (size_t)n * NOUT, cudaMemcpyHostToDevice, st), "copy");
    double h[2 * (NIN + NOUT)];
    if (rc == MS_OK) {
        k_col_stats<<<NIN, 256, 0, st>>>(Xd, n, NIN, 1e-12, sd);
        k_col_stats<<<NOUT, 256, 0, st>>>(Yd, n, NOUT, 1e-12, sd + 2 * NIN);
        rc = ck(cudaGetLastError(), "k_col_stats");
    }
    if (rc == MS_OK) rc = ck(cudaMemcpyAsync(h, sd, sizeof(h), cudaMemcpyDeviceToHost, st), "copy");
    if (rc == MS_OK) rc = ck(cudaStreamSynchronize(st), "sync");
    if (st) cudaStreamSynchronize(st);
    cudaFree(Xd);
    cudaFree(Yd);
    cudaFree(sd);
    if (st) cudaStreamDestroy(st);
    if (rc != MS_OK) return rc;
    // packed as ms_mlp_create reads it: mu_x, sd_x, mu_y, sd_y
    for (int i = 0; i < 2 * NIN; i++) norm[i] = (float)h[i];
    for (int i = 0; i < 2 * NOUT; i++) norm[2 * NIN + i] = (float)h[2 * NIN + i];
    return MS_OK;
}

void ms_mlp_free(ms_mlp *m)
{
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    for (void *p : m->allocs) cudaFree(p);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
}

// device-pointer forward used by the model's hybrid step: X [n][16] raw -> Y [n][4]
int ms_mlp_forward_device(ms_mlp *m, const float *X, int64_t n, float *Y, void *stream)
{
    if (!m || (n > 0 && (!X || !Y))) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (m->engine == 1) {
        TcArgs a{};
        a.X = X;
        a.Y = Y;
        a.n = n;
        for (int l = 0; l < 4; l++) {
            a.W[l] = m->L[l].Wc;
            a.b[l] = m->L[l].b;
        }
        a.mu_x = m->mu_x;
        a.sd_x = m->sd_x;
        a.mu_y = m->mu_y;
        a.sd_y = m->sd_y;
        a.err = m->tc_err;
        // two 107 KB CTAs fit an SM
        return ck(launch_mlp_forward_tc(a, 2 * m->sm_count, stream ? (cudaStream_t)stream : m->st), "tcgen05 forward");
    }
    cudaStream_t keep = m->st;
    if (stream) m->st = (cudaStream_t)stream;
    int rc = MS_OK;
    for (int64_t s0 = 0; s0 < n && rc == MS_OK; s0 += m->max_batch) {
        const int B = (int)std::min<int64_t>(m->max_batch, n - s0), Bp = pad8(B);
        k_prep_input<<<(Bp + 255) / 256, 256, 0, m->st>>>(X + s0 * NIN, B, Bp, m->mu_x, m->sd_x, m->xh, m->xht);
        rc = ck(forward(m, Bp), "forward");
        if (rc == MS_OK) k_denorm<<<(B + 255) / 256, 256, 0, m->st>>>(m->yp, B, m->mu_y, m->sd_y, Y + s0 * NOUT);
        if (rc == MS_OK) rc = ck(cudaGetLastError(), "denorm");
    }
    m->st = keep;
    return rc;
}

int ms_mlp_predict(ms_mlp *m, const float *X, int64_t n, float *Y)
{
    if (!m || n < 0 || (n > 0 && (!X || !Y))) return ms_closure_fail(MS_ERR_ARG, "bad argument");
    for (int64_t s0 = 0; s0 < n; s0 += m->max_batch) {
        const int B = (int)std::min<int64_t>(m->max_batch, n - s0);
        CKC(cudaMemcpyAsync(m->X, X + s0 * NIN, sizeof(float) * B * NIN, cudaMemcpyHostToDevice, m->st));
        int rc = ms_mlp_forward_device(m, m->X, B, m->yout, nullptr);
        if (rc) return rc;
        CKC(cudaMemcpyAsync(Y + s0 * NOUT, m->yout, sizeof(float) * B * NOUT, cudaMemcpyDeviceToHost, m->st));
        CKC(cudaStreamSynchronize(m->st));
    }
    return ms_mlp_check(m);
}

int ms_mlp_set_engine(ms_mlp *m, int32_t engine)
{
    if (!m) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (engine != 0 && engine != 1) return ms_closure_fail(MS_ERR_ARG, "engine must be 0 or 1");
    CKC(cudaStreamSynchronize(m->st));
    m->engine = engine;
    return MS_OK;
}

int ms_mlp_check(ms_mlp *m)
{
    if (!m) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    int err = 0;
    CKC(cudaMemcpy(&err, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CKC(cudaMemset(m->tc_err, 0, sizeof(int)));
        return ms_closure_fail(MS_ERR_TIMEOUT, "a wait on the tensor cores ran out in the closure network");
    }
    return MS_OK;
}

static AdamHyper adam_hyper(const ms_mlp *m, float lr)
{
    AdamHyper h;
    h.lr = lr;
    h.beta1 = 0.9f;
    h.beta2 = 0.999f;
    h.eps = 1e-8f;
    h.tstep = m->d_t;
    return h;
}

// the gradients of the batch (X, Y) already on the device into the layers'
// gW, gb (which hold zeros) and its loss added to m->loss: on engine 1 the
// two tcgen05 kernels, on engine 0 the mma.sync GEMMs
static cudaError_t batch_grads(ms_mlp *m, const float *Xd, const float *Yd, int B, bool tick)
{
    const int Bp = pad8(B);
    if (m->engine == 1) {
        TrainArgs a{};
        a.X = Xd;
        a.Y = Yd;
        a.B = B;
        a.Bp = Bp;
        for (int l = 0; l < 4; l++) {
            a.W[l] = m->L[l].Wc;
            a.Wt[l] = m->L[l].Wtc;
            a.b[l] = m->L[l].b;
        }
        a.mu_x = m->mu_x;
        a.sd_x = m->sd_x;
        a.mu_y = m->mu_y;
        a.sd_y = m->sd_y;
        a.xt = m->xht;
        for (int l = 0; l < 3; l++) {
            a.Ht[l] = m->Ht[l];
            a.dZt[l] = m->dZt[l];
        }
        a.dyt = m->dyt;
        a.loss = m->loss;
        a.tick = tick ? m->d_t : nullptr;
        a.err = m->tc_err;
        cudaError_t e = launch_train_tile_tc(a, m->sm_count, m->st);
        if (e != cudaSuccess) return e;
        WgradArgs w{};
        w.njob = 4;
        w.K = Bp;
        w.err = m->tc_err;
        for (int l = 0; l < 4; l++) {
            WgradJob &J = w.job[l];
            J.M = LOUT[l];
            J.nin = LIN[l];
            J.ldw = LKIN[l];
            J.A = l == 3 ? m->dyt : m->dZt[l];
            J.B = l == 0 ? m->xht : m->Ht[l - 1];
            J.gW = m->L[l].gW;
            J.gb = m->L[l].gb;
        }
        return launch_wgrad_tc(w, m->sm_count, m->st);
    }
    k_prep_input<<<(Bp + 255) / 256, 256, 0, m->st>>>(Xd, B, Bp, m->mu_x, m->sd_x, m->xh, m->xht);
    const float *keepY = m->Y;
    m->Y = const_cast<float *>(Yd);
    cudaError_t e = forward(m, Bp);
    if (e == cudaSuccess) e = backward(m, B, Bp);
    m->Y = const_cast<float *>(keepY);
    if (e == cudaSuccess && tick) k_tick<<<1, 1, 0, m->st>>>(m->d_t);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// gradients and loss back to zero
static cudaError_t zero_grads(ms_mlp *m)
{
    cudaError_t e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->st);
    for (int l = 0; l < 4 && e == cudaSuccess; l++) {
        e = cudaMemsetAsync(m->L[l].gW, 0, sizeof(float) * m->L[l].nop * m->L[l].kin, m->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->L[l].gb, 0, sizeof(float) * m->L[l].nout, m->st);
    }
    return e;
}

static int gather_grads(ms_mlp *m, float *grads)
{
    size_t off = 0;
    std::vector<float> tmp;
    for (int l = 0; l < 4; l++) {
        const LayerDev &L = m->L[l];
        tmp.resize((size_t)L.nop * L.kin);
        CKC(cudaMemcpyAsync(tmp.data(), L.gW, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, m->st));
        CKC(cudaMemcpyAsync(grads + off + (size_t)L.nout * L.nin, L.gb, sizeof(float) * L.nout, cudaMemcpyDeviceToHost,
                            m->st));
        CKC(cudaStreamSynchronize(m->st));
        for (int o = 0; o < L.nout; o++)
            for (int k = 0; k < L.nin; k++) grads[off + (size_t)o * L.nin + k] = tmp[(size_t)o * L.kin + k];
        off += (size_t)L.nout * L.nin + L.nout;
    }
    return MS_OK;
}

int ms_mlp_grad(ms_mlp *m, const float *X, const float *Y, int64_t n, float *grads, double *loss)
{
    if (!m || !X || !Y || !grads) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (n < 1 || n > m->max_batch) return ms_closure_fail(MS_ERR_ARG, "n must be in [1, max_batch]");
    const int B = (int)n;
    CKC(cudaMemcpyAsync(m->X, X, sizeof(float) * B * NIN, cudaMemcpyHostToDevice, m->st));
    CKC(cudaMemcpyAsync(m->Y, Y, sizeof(float) * B * NOUT, cudaMemcpyHostToDevice, m->st));
    CKC(zero_grads(m));
    CKC(batch_grads(m, m->X, m->Y, B, false));
    if (loss) CKC(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    CKC(cudaStreamSynchronize(m->st));
    int rc = gather_grads(m, grads);
    if (rc == MS_OK) rc = ck(zero_grads(m), "memset");
    return rc ? rc : ms_mlp_check(m);
}

int ms_mlp_get_params(ms_mlp *m, float *params)
{
    if (!m || !params) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    size_t off = 0;
    for (int l = 0; l < 4; l++) {
        const LayerDev &L = m->L[l];
        const size_t nw = (size_t)L.nout * L.nin;
        CKC(cudaMemcpyAsync(params + off, L.W, sizeof(float) * nw, cudaMemcpyDeviceToHost, m->st));
        off += nw;
        CKC(cudaMemcpyAsync(params + off, L.b, sizeof(float) * L.nout, cudaMemcpyDeviceToHost, m->st));
        off += L.nout;
    }
    CKC(cudaStreamSynchronize(m->st));
    return MS_OK;
}

// one Adam step on the gradients of the batch (X, Y) already on the device;
// the batch's loss (times B) into eloss[*d_ep] if eloss is not null
static int train_step(ms_mlp *m, const float *Xd, const float *Yd, int B, float lr, double *eloss)
{
    CKC(batch_grads(m, Xd, Yd, B, true));
    AdamAll A{};
    A.off[0] = 0;
    for (int l = 0; l < 4; l++) {
        A.L[l] = m->L[l];
        A.off[l + 1] = A.off[l] + m->L[l].nout * m->L[l].nin + m->L[l].nout;
    }
    A.loss = m->loss;
    A.eloss = eloss;
    A.ep = m->d_ep;
    A.B = B;
    k_adam<<<(A.off[4] + 255) / 256, 256, 0, m->st>>>(A, adam_hyper(m, lr));
    return ck(cudaGetLastError(), "adam");
}

int ms_mlp_step(ms_mlp *m, const float *X, const float *Y, int64_t n, float lr)
{
    if (!m || !X || !Y) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (n < 1 || n > m->max_batch) return ms_closure_fail(MS_ERR_ARG, "n must be in [1, max_batch]");
    CKC(cudaMemcpyAsync(m->X, X, sizeof(float) * n * NIN, cudaMemcpyHostToDevice, m->st));
    CKC(cudaMemcpyAsync(m->Y, Y, sizeof(float) * n * NOUT, cudaMemcpyHostToDevice, m->st));
    CKC(zero_grads(m));
    int rc = train_step(m, m->X, m->Y, (int)n, lr, nullptr);
    if (rc) return rc;
    CKC(cudaStreamSynchronize(m->st));
    return ms_mlp_check(m);
}

int ms_mlp_train(ms_mlp *m, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, double *loss_per_epoch)
{
    if (!m || !X || !Y) return ms_closure_fail(MS_ERR_ARG, "NULL argument");
    if (n < 1 || epochs < 0 || batch < 8 || batch > m->max_batch || !(lr > 0.0f))
        return ms_closure_fail(MS_ERR_ARG, "need n >= 1, epochs >= 0, 8 <= batch <= max_batch, lr > 0");
    if (n > (int64_t)1 << 30) return ms_closure_fail(MS_ERR_ARG, "at most 2^30 samples");
    // the training set on the device once; each epoch gathers it in the
    // epoch's order on the device and replays one captured graph of its
    // batches; the per-epoch losses stay on the device until the end
    float *Xd = nullptr, *Yd = nullptr, *Xs = nullptr, *Ys = nullptr;
    double *el = nullptr;
    std::vector<void *> loc;
    auto dm = [&](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) loc.push_back(*p);
        return e;
    };
    cudaGraphExec_t gexec = nullptr;
    auto cleanup = [&]() {
        if (gexec) cudaGraphExecDestroy(gexec);
        for (void *p : loc) cudaFree(p);
    };
    cudaError_t e;
    if ((e = dm((void **)&Xd, sizeof(float) * n * NIN)) || (e = dm((void **)&Yd, sizeof(float) * n * NOUT)) ||
        (e = dm((void **)&Xs, sizeof(float) * n * NIN)) || (e = dm((void **)&Ys, sizeof(float) * n * NOUT)) ||
        (e = dm((void **)&el, sizeof(double) * (epochs > 0 ? epochs : 1)))) {
        cleanup();
        return ck(e, "cudaMalloc");
    }
    int rc = MS_OK;
    auto run = [&](cudaError_t x, const char *what) {
        if (rc == MS_OK) rc = ck(x, what);
    };
    run(cudaMemcpyAsync(Xd, X, sizeof(float) * n * NIN, cudaMemcpyHostToDevice, m->st), "copy");
    run(cudaMemcpyAsync(Yd, Y, sizeof(float) * n * NOUT, cudaMemcpyHostToDevice, m->st), "copy");
    run(cudaMemsetAsync(el, 0, sizeof(double) * (epochs > 0 ? epochs : 1), m->st), "memset");
    run(zero_grads(m), "memset");
    // Feistel domain 4^h >= n
    int h = 1;
    while (((int64_t)1 << (2 * h)) < n) h++;
    uint64_t sm = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto next = [&]() {   // SplitMix64: the epochs' keys
        sm += 0x9E3779B97F4A7C15ull;
        uint64_t z = sm;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    // one epoch's batches (a ragged last batch below 8 samples is dropped)
    int64_t used = 0;
    auto batches = [&]() -> int {
        used = 0;
        for (int64_t s0 = 0; s0 < n; s0 += batch) {
            const int B = (int)std::min<int64_t>(batch, n - s0);
            if (B < 8) break;
            const int r = train_step(m, Xs + s0 * NIN, Ys + s0 * NOUT, B, lr, loss_per_epoch ? el : nullptr);
            if (r) return r;
            used += B;
        }
        return ck(cudaGetLastError(), "batch");
    };
    if (rc == MS_OK && epochs > 0) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int r = batches();
            const cudaError_t ee = cudaStreamEndCapture(m->st, &g);
            if (r == MS_OK && ee == cudaSuccess && g && cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess)
                gexec = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();   // a capture that failed leaves the direct launches below
    }
    for (int ep = 0; ep < epochs && rc == MS_OK; ep++) {
        const uint64_t k1 = next(), k2 = next();
        const uint4 key = make_uint4((uint32_t)k1, (uint32_t)(k1 >> 32), (uint32_t)k2, (uint32_t)(k2 >> 32));
        k_gather_epoch<<<(unsigned)((n + 255) / 256), 256, 0, m->st>>>(Xd, Yd, n, h, key, Xs, Ys);
        k_set_epoch<<<1, 1, 0, m->st>>>(m->d_ep, ep);
        run(cudaGetLastError(), "gather");
        if (rc) break;
        if (gexec) run(cudaGraphLaunch(gexec, m->st), "epoch graph");
        else rc = batches();
    }
    if (rc == MS_OK && loss_per_epoch && epochs > 0) {
        std::vector<double> hl(epochs);
        run(cudaMemcpyAsync(hl.data(), el, sizeof(double) * epochs, cudaMemcpyDeviceToHost, m->st), "copy");
        run(cudaStreamSynchronize(m->st), "sync");
        if (rc == MS_OK)
            for (int ep = 0; ep < epochs; ep++) loss_per_epoch[ep] = used ? hl[ep] / (double)used : 0.0;
    }
    if (rc == MS_OK) rc = ck(cudaStreamSynchronize(m->st), "sync");
    cleanup();
    return rc == MS_OK ? ms_mlp_check(m) : rc;
}

}  // extern "C"
