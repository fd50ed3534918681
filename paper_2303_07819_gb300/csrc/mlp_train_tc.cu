// mlp_train_tc.cu -- one Adam batch of the closure network on the tcgen05
// tensor cores in two kernels (the Adam update is a third, in closure.cu).
//
// k_train_tile_tc: a persistent CTA of 256 threads per SM keeps the four
// forward weight images and the three transposed ones of the backward pass
// in shared memory (140 KB, staged by seven cp.async.bulk copies) and takes
// tiles of 128 samples, two threads per sample (each takes half of a layer's
// units in the epilogues).  For each tile it runs seven
// tcgen05.mma chains, each into the same 128-column FP32 accumulator in
// tensor memory:
//   forward   h_l = tanh(W_l h_{l-1} + b_l), l = 0, 1, 2;  y = W_3 h_2 + b_3
//   loss      r = y - (target - mu_y) / sd_y,  dL/dy = 2 r / (4 B)
//   backward  dz_{l-1} = (W_l^T dz_l) (1 - h_{l-1}^2), l = 3, 2, 1 (dz_3 = dL/dy)
// Each chain's epilogue reads the sample's row (tcgen05.ld) and writes the
// next chain's BF16 operand over the last one in shared memory.  The hidden
// activations also stay in tensor memory for the tanh derivative of the
// backward pass (all 512 columns: one CTA per SM), and the transposed
// activations and dz go to global memory for the weight gradients, staged in
// shared memory and written while the next chain's MMAs run.
//
// k_wgrad_tc: the weight gradients dz_l^T h_{l-1} of the four layers as one
// launch of 128 x 64 tcgen05 tiles (tc_gemm.cuh) over k slices of the batch,
// added atomically; a row of ones appended to h_{l-1} gives the bias gradient
// (the sum of dz_l over the batch) in the same products.
//
// Every wait on an mbarrier is bounded: a wait that runs out sets the error
// word, waits once more (bounded) for the work in flight, and the CTA frees
// its tensor memory and stops.
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"
#include "mlp_tc.cuh"
#include "tc_gemm.cuh"

namespace msd {

namespace {

using namespace tcx;
typedef __nv_bfloat16 bf16;

constexpr int TR_T = 128;          // samples per tile = MMA M = tensor-memory lanes
constexpr int TR_THREADS = 256;    // two threads per sample: warps w and w + 4 share lanes 32 (w % 4) ..
constexpr int TR_NH = 128;         // hidden width
constexpr int TR_KIN = 16;         // input features
constexpr int TR_NO = 16;          // output layer padded to the smallest N (forward) and K (backward)
constexpr int TR_COLS = 512;       // tensor-memory columns: the accumulator, then h_0, h_1, h_2 (FP32)

struct TrSmem {
    bf16 W0[TR_NH * TR_KIN];       // forward images [out][in]: 128 x 16
    bf16 W1[TR_NH * TR_NH];        // 128 x 128
    bf16 W2[TR_NH * TR_NH];
    bf16 W3[TR_NO * TR_NH];        // 16 x 128, rows 4-15 zero
    bf16 T1[TR_NH * TR_NH];        // backward images W_l^T [in][out]: 128 x 128
    bf16 T2[TR_NH * TR_NH];
    bf16 T3[TR_NH * TR_NO];        // 128 x 16, columns 4-15 zero
    bf16 A[TR_T * TR_NH];          // the tile's operand, [128][K] for K = 16 or 128
    bf16 Tr[TR_NH * TR_T];         // a layer's output transposed, [unit][sample], on its way to global memory
    float b[3][TR_NH], b3[TR_NO];
    float mux[TR_KIN], sdx[TR_KIN], muy[4], sdy[4];
    double lsum[TR_THREADS / 32];
    unsigned long long bar;        // mbarrier of the MMA chains
    unsigned long long wbar;       // mbarrier of the weights' bulk copies
    uint32_t tbase;
};

__global__ void __launch_bounds__(TR_THREADS) k_train_tile_tc(TrainArgs a)
{
    extern __shared__ __align__(128) unsigned char tr_raw[];
    TrSmem &S = *reinterpret_cast<TrSmem *>(tr_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // this thread's sample (tensor-memory lane) and half of the units
    const int r = 32 * (warp & 3) + lane, half = warp >> 2;
    const uint32_t wbar = smem_u32(&S.wbar);
    constexpr uint32_t SQ = TR_NH * TR_NH * 2, SM16 = TR_NH * TR_KIN * 2;   // bytes of the images
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(wbar), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(wbar), "r"(4 * SQ + 3 * SM16) : "memory");
        bulk_g2s(smem_u32(S.W0), a.W[0], SM16, wbar);
        bulk_g2s(smem_u32(S.W1), a.W[1], SQ, wbar);
        bulk_g2s(smem_u32(S.W2), a.W[2], SQ, wbar);
        bulk_g2s(smem_u32(S.W3), a.W[3], SM16, wbar);
        bulk_g2s(smem_u32(S.T1), a.Wt[1], SQ, wbar);
        bulk_g2s(smem_u32(S.T2), a.Wt[2], SQ, wbar);
        bulk_g2s(smem_u32(S.T3), a.Wt[3], SM16, wbar);
    }
    for (int i = t; i < 3 * TR_NH; i += TR_THREADS) S.b[i / TR_NH][i % TR_NH] = a.b[i / TR_NH][i % TR_NH];
    if (t < TR_NO) S.b3[t] = t < 4 ? a.b[3][t] : 0.0f;
    if (t < TR_KIN) {
        S.mux[t] = a.mu_x[t];
        S.sdx[t] = a.sd_x[t];
    }
    if (t < 4) {
        S.muy[t] = a.mu_y[t];
        S.sdy[t] = a.sd_y[t];
    }
    const uint32_t bar = smem_u32(&S.bar);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S.tbase)), "r"(TR_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    bool ok = __syncthreads_and(bar_wait(wbar, 0u) ? 1 : 0) != 0;
    const bool weights_ok = ok;
    const uint32_t tmem = S.tbase;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t sA = smem_u32(S.A);
    unsigned char *Ab = reinterpret_cast<unsigned char *>(S.A);
    uint32_t phase = 0;
    const size_t Bp = (size_t)a.Bp;
    const int cbeg = half * (TR_NH / 2), cend = cbeg + TR_NH / 2;   // this thread's units

    // S.Tr -> rows of a transposed [units][Bp] array from column m0 on (its
    // samples below Bp), 16-byte pieces
    bf16 *tr_dst = nullptr;
    int tr_m0 = 0;
    auto flush_tr = [&]() {
        if (!tr_dst) return;
#pragma unroll 4
        for (int i = 0; i < TR_NH * TR_T / 8 / TR_THREADS; i++) {
            const int q = t + i * TR_THREADS, n = q / (TR_T / 8), j = q % (TR_T / 8);
            if (tr_m0 + 8 * j < a.Bp)
                *reinterpret_cast<uint4 *>(tr_dst + (size_t)n * Bp + tr_m0 + 8 * j) =
                    *reinterpret_cast<const uint4 *>(&S.Tr[n * TR_T + 8 * j]);
        }
        tr_dst = nullptr;
    };

    // one chain D = A B^T (M = 128, N, K) into the accumulator; the previous
    // layer's transposed output goes to global memory while the MMAs run.
    // The same outcome in every thread.
    auto chain = [&](uint32_t sB, int K, int N) -> bool {
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (t == 0) {
            const uint32_t id = idesc_bf16(TR_T, N);
            for (int kk = 0; kk < K / 16; kk++)
                mma_issue(tmem, sdesc(sA + kk * 256, 128, 16 * K), sdesc(sB + kk * 256, 128, 16 * K), id,
                          kk > 0 ? 1u : 0u);
            mma_commit(bar);
        }
        flush_tr();
        const bool ok2 = __syncthreads_and(bar_wait(bar, phase) ? 1 : 0) != 0;
        if (ok2) {
            phase ^= 1u;
            fence_after();
        }
        return ok2;
    };

    const int ntiles = (a.Bp + TR_T - 1) / TR_T;
    const float inv4B = 1.0f / (4.0f * (float)a.B);
    double lsum = 0.0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int m0 = tile * TR_T, m = m0 + r;
        const bool inB = m < a.B, inBp = m < a.Bp;
        // z-scored inputs: the first operand (K = 16) and their transpose;
        // each half of the threads takes 8 features
        {
            const int f0 = 8 * half;
            float x[8];
            if (inB) {
                const float4 *xp = reinterpret_cast<const float4 *>(a.X + (size_t)m * TR_KIN + f0);
                const float4 u0 = xp[0], u1 = xp[1];
                x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
#pragma unroll
                for (int e = 0; e < 8; e++) x[e] = (x[e] - S.mux[f0 + e]) / S.sdx[f0 + e];
            } else {
#pragma unroll
                for (int e = 0; e < 8; e++) x[e] = 0.0f;
            }
            __align__(16) bf16 h[8];
#pragma unroll
            for (int e = 0; e < 8; e++) h[e] = __float2bfloat16_rn(x[e]);
            *reinterpret_cast<uint4 *>(Ab + core_off(r, f0, TR_KIN)) = *reinterpret_cast<const uint4 *>(h);
            if (inBp)
#pragma unroll
                for (int e = 0; e < 8; e++) a.xt[(size_t)(f0 + e) * Bp + m] = h[e];
        }
        // hidden layers: h_l to the next operand, to tensor memory (FP32 of
        // the BF16 value, for the backward pass) and transposed to S.Tr
        const uint32_t sW[3] = {smem_u32(S.W0), smem_u32(S.W1), smem_u32(S.W2)};
        for (int l = 0; l < 3 && ok; l++) {
            ok = chain(sW[l], l == 0 ? TR_KIN : TR_NH, TR_NH);
            if (!ok) break;
            // this thread's 64 columns: four loads in flight, one wait
            uint32_t acc[4][16];
            __syncwarp();
#pragma unroll
            for (int g = 0; g < 4; g++) tmem_ld16_issue(lane_addr + (uint32_t)(cbeg + 16 * g), acc[g]);
#pragma unroll
            for (int g = 0; g < 4; g++) tmem_ld_wait(acc[g]);
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const int c0 = cbeg + 16 * g;
                float v[16];
                __align__(16) bf16 h[16];
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    h[e] = __float2bfloat16_rn(tanh_sfu(__uint_as_float(acc[g][e]) + S.b[l][c0 + e]));
                    v[e] = __bfloat162float(h[e]);
                    S.Tr[(c0 + e) * TR_T + r] = h[e];
                }
                tmem_st16(lane_addr + (uint32_t)(TR_NH * (l + 1) + c0), v);
                *reinterpret_cast<uint4 *>(Ab + core_off(r, c0, TR_NH)) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(Ab + core_off(r, c0 + 8, TR_NH)) = *reinterpret_cast<const uint4 *>(h + 8);
            }
            tmem_st_wait();
            tr_dst = a.Ht[l];
            tr_m0 = m0;
            fence_before();
        }
        if (!ok) break;
        // output layer and the loss: dL/dy is the first backward operand
        // (K = 16), written by the first half of the threads
        ok = chain(smem_u32(S.W3), TR_NH, TR_NO);
        if (!ok) break;
        {
            float v[16];
            tmem_ld16(lane_addr, v);
            if (half == 0) {
                __align__(16) bf16 g[16];
#pragma unroll
                for (int e = 0; e < 16; e++) g[e] = __float2bfloat16_rn(0.0f);
                if (inB) {
                    const float4 y = *reinterpret_cast<const float4 *>(a.Y + (size_t)m * 4);
                    const float yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int o = 0; o < 4; o++) {
                        const float res = v[o] + S.b3[o] - (yv[o] - S.muy[o]) / S.sdy[o];
                        lsum += (double)res * res;
                        g[o] = __float2bfloat16_rn(2.0f * res * inv4B);
                    }
                }
                *reinterpret_cast<uint4 *>(Ab + core_off(r, 0, TR_NO)) = *reinterpret_cast<const uint4 *>(g);
                *reinterpret_cast<uint4 *>(Ab + core_off(r, 8, TR_NO)) = *reinterpret_cast<const uint4 *>(g + 8);
                if (inBp)
#pragma unroll
                    for (int o = 0; o < 4; o++) a.dyt[(size_t)o * Bp + m] = g[o];
            }
            fence_before();
        }
        // backward through layers 3, 2, 1: dz of the hidden layers 2, 1, 0
        const uint32_t sT[4] = {0u, smem_u32(S.T1), smem_u32(S.T2), smem_u32(S.T3)};
        for (int l = 3; l >= 1 && ok; l--) {
            ok = chain(sT[l], l == 3 ? TR_NO : TR_NH, TR_NH);
            if (!ok) break;
#pragma unroll 1
            for (int c1 = cbeg; c1 < cend; c1 += 32) {
                // two groups of 16 columns and their h_{l-1}: four loads in flight, one wait
                uint32_t acc[2][16], hh[2][16];
                __syncwarp();
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    tmem_ld16_issue(lane_addr + (uint32_t)(c1 + 16 * g), acc[g]);
                    tmem_ld16_issue(lane_addr + (uint32_t)(TR_NH * l + c1 + 16 * g), hh[g]);
                }
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    tmem_ld_wait(acc[g]);
                    tmem_ld_wait(hh[g]);
                }
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    const int c0 = c1 + 16 * g;
                    __align__(16) bf16 d[16];
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const float h = __uint_as_float(hh[g][e]);
                        d[e] = __float2bfloat16_rn(__uint_as_float(acc[g][e]) * (1.0f - h * h));
                        S.Tr[(c0 + e) * TR_T + r] = d[e];
                    }
                    if (l > 1) {
                        *reinterpret_cast<uint4 *>(Ab + core_off(r, c0, TR_NH)) = *reinterpret_cast<const uint4 *>(d);
                        *reinterpret_cast<uint4 *>(Ab + core_off(r, c0 + 8, TR_NH)) =
                            *reinterpret_cast<const uint4 *>(d + 8);
                    }
                }
            }
            tr_dst = a.dZt[l - 1];
            tr_m0 = m0;
            fence_before();
        }
        // dz_0 is the tile's last output: to global memory before S.Tr is reused
        __syncthreads();
        flush_tr();
    }
    // the loss: one atomic per CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.lsum[warp] = lsum;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < TR_THREADS / 32; w++) s += S.lsum[w];
        if (s != 0.0) atomicAdd(a.loss, s / (4.0 * (double)a.B));
        if (blockIdx.x == 0 && a.tick) *a.tick += 1;
    }
    if (!ok) {
        if (t == 0) atomicOr(a.err, 1);
        if (weights_ok) bar_wait(bar, phase);   // the chain in flight, if it still completes
        else bar_wait(wbar, 0u);                // the copies in flight, if they still complete
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TR_COLS));
}

// The weight-gradient jobs: blockIdx.x runs over every job's 64-column tiles
// of [nin + 1] columns (the last one the row of ones), blockIdx.z over the
// k slices of kchunk samples.
__global__ void __launch_bounds__(TCG_T) k_wgrad_tc(WgradArgs a, int kchunk)
{
    extern __shared__ __align__(128) unsigned char wg_raw[];
    TcgSmem &S = *reinterpret_cast<TcgSmem *>(wg_raw);
    const int t = threadIdx.x, warp = t >> 5;
    int bx = blockIdx.x, j = 0;
    for (; j < a.njob; j++) {
        const int nt = (a.job[j].nin + 1 + TCG_NT - 1) / TCG_NT;
        if (bx < nt) break;
        bx -= nt;
    }
    if (j == a.njob) return;   // uniform over the CTA: before any barrier
    const WgradJob &J = a.job[j];
    const int N = J.nin + 1, n0 = bx * TCG_NT;
    const int kbeg = blockIdx.z * kchunk, kend = min(a.K, kbeg + kchunk);
    const int Np = (min(TCG_NT, N - n0) + 15) / 16 * 16;
    const uint32_t tmem = tcg_init(S);
    TcgState st;
    const bool ok = tcg_mainloop(S, tmem, st, J.M, N, kbeg, kend, 0, n0, J.A, a.K, J.B, a.K, J.nin);
    if (ok && kend > kbeg) {
        const int m = t;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float v[16];
            tmem_ld16(lane_addr + c0, v);
            if (m >= J.M) continue;
            const int nb = n0 + c0;
            float *p = J.gW + (size_t)m * J.ldw + nb;
            if (nb + 16 <= J.nin) {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    atomicAdd(reinterpret_cast<float4 *>(p + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
            } else {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    if (nb + i < J.nin) atomicAdd(p + i, v[i]);
                    else if (nb + i == J.nin) atomicAdd(J.gb + m, v[i]);
                }
            }
        }
    }
    tcg_finish(S, tmem, st, ok, a.err);
}

}  // namespace

cudaError_t mlp_train_tc_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_train_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcgSmem));
}

cudaError_t launch_train_tile_tc(const TrainArgs &a, int sm_count, cudaStream_t st)
{
    if (a.Bp <= 0) return cudaSuccess;
    const int ntiles = (a.Bp + TR_T - 1) / TR_T;
    const int grid = ntiles < sm_count ? ntiles : sm_count;
    k_train_tile_tc<<<grid, TR_THREADS, sizeof(TrSmem), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_tc(const WgradArgs &a, int sm_count, cudaStream_t st)
{
    if (a.K <= 0 || a.njob <= 0) return cudaSuccess;
    int tiles = 0;
    for (int j = 0; j < a.njob; j++) tiles += (a.job[j].nin + 1 + TCG_NT - 1) / TCG_NT;
    const int chunks = (a.K + TCG_BK - 1) / TCG_BK;
    int ks = (2 * sm_count + tiles - 1) / tiles;
    ks = ks < 1 ? 1 : (ks > chunks ? chunks : ks);
    const int kchunk = ((a.K + ks - 1) / ks + TCG_BK - 1) / TCG_BK * TCG_BK;
    dim3 grid(tiles, 1, (a.K + kchunk - 1) / kchunk);
    k_wgrad_tc<<<grid, TCG_T, sizeof(TcgSmem), st>>>(a, kchunk);
    return cudaGetLastError();
}

}  // namespace msd
