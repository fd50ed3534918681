// mlp_tc.cu -- closure network inference on the fifth-generation tensor
// cores (tcgen05): one persistent kernel for the 16 -> 128 -> 128 -> 128 -> 4
// tanh MLP.
//
// A CTA of 128 threads keeps all four BF16 weight matrices in shared memory
// and takes tiles of 128 cells, a thread per cell.  Each layer is a chain of
// tcgen05.mma.kind::f16 (M = 128 cells, N = 128 units or 16 for the padded
// output layer, K = 16 per instruction) issued by one thread: A is the
// tile's activations, B the layer's weights [out][in], both K-major BF16 in
// shared memory, D the FP32 accumulator in tensor memory (128 lanes = the
// tile's cells, one column per unit).  A commit to an mbarrier marks the
// chain done; every thread then reads its cell's row with tcgen05.ld, adds
// the bias, applies tanh (the special-function unit's tanh.approx) and writes
// the next layer's BF16 operand in place.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8 x 16-byte "core matrices" (8 rows, 8 BF16 along K), core matrix (i, j)
// of an R x K operand at byte (i K/8 + j) 128, so the descriptor's leading
// byte offset (next core matrix along K) is 128 and its stride byte offset
// (next 8 rows) is 16 K.
//
// The weights arrive by four cp.async.bulk copies of their images (kept in
// global memory in this layout by the trainer) completing on an mbarrier.
// Every wait on an mbarrier is bounded: a wait that runs out sets the error
// word, waits once more (bounded) for the work in flight, and the CTA frees
// its tensor memory and stops.
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"
#include "mlp_tc.cuh"
#include "tc_ptx.cuh"

namespace msd {

namespace {

using namespace tcx;
typedef __nv_bfloat16 bf16;

constexpr int TC_T = 128;          // threads = cells per tile = MMA M
constexpr int TC_NH = 128;         // hidden width
constexpr int TC_KIN = 16;         // input features
constexpr int TC_NO = 16;          // output layer padded to the smallest N
constexpr int TC_COLS = 128;       // tensor-memory columns held (power of 2, >= 32)

struct TcSmem {
    bf16 W0[TC_NH * TC_KIN];       // [128][16]
    bf16 W1[TC_NH * TC_NH];        // [128][128]
    bf16 W2[TC_NH * TC_NH];
    bf16 W3[TC_NO * TC_NH];        // [16][128], rows 4-15 zero
    bf16 A[TC_T * TC_NH];          // the tile's operand, [128][K] for K = 16 or 128
    float b[3][TC_NH], b3[TC_NO];
    float mux[TC_KIN], sdx[TC_KIN], muy[4], sdy[4];
    unsigned long long bar;        // mbarrier of the MMA chains
    unsigned long long wbar;       // mbarrier of the weights' bulk copies
    uint32_t tbase;                // tensor-memory address from tcgen05.alloc
};

__global__ void __launch_bounds__(TC_T) k_mlp_forward_tc(TcArgs a)
{
    extern __shared__ __align__(128) unsigned char tc_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw);
    const int t = threadIdx.x, warp = t >> 5;
    // the weight images by four bulk copies on their own mbarrier
    const uint32_t wbar = smem_u32(&S.wbar);
    constexpr uint32_t wbytes[4] = {TC_NH * TC_KIN * 2, TC_NH * TC_NH * 2, TC_NH * TC_NH * 2, TC_NO * TC_NH * 2};
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(wbar), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(wbar), "r"(wbytes[0] + wbytes[1] + wbytes[2] + wbytes[3]) : "memory");
        bulk_g2s(smem_u32(S.W0), a.W[0], wbytes[0], wbar);
        bulk_g2s(smem_u32(S.W1), a.W[1], wbytes[1], wbar);
        bulk_g2s(smem_u32(S.W2), a.W[2], wbytes[2], wbar);
        bulk_g2s(smem_u32(S.W3), a.W[3], wbytes[3], wbar);
    }
    for (int i = t; i < 3 * TC_NH; i += TC_T) S.b[i / TC_NH][i % TC_NH] = a.b[i / TC_NH][i % TC_NH];
    if (t < TC_NO) S.b3[t] = t < 4 ? a.b[3][t] : 0.0f;
    if (t < TC_KIN) {
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
                     :: "r"(smem_u32(&S.tbase)), "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // the weights in shared memory (every thread waits; the same outcome for all)
    bool ok = __syncthreads_and(bar_wait(wbar, 0u) ? 1 : 0) != 0;
    const uint32_t tmem = S.tbase;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
    const uint32_t sA = smem_u32(S.A), sW[4] = {smem_u32(S.W0), smem_u32(S.W1), smem_u32(S.W2), smem_u32(S.W3)};
    uint32_t phase = 0;
    const bool weights_ok = ok;
    const int ntiles = (a.n + TC_T - 1) / TC_T;
    unsigned char *Ab = reinterpret_cast<unsigned char *>(S.A);

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long row = (long long)tile * TC_T + t;
        // z-scored features -> BF16 operand of layer 0 (K = 16)
        {
            float x[TC_KIN];
#pragma unroll
            for (int f = 0; f < TC_KIN; f++)
                x[f] = row < a.n ? (a.X[row * TC_KIN + f] - S.mux[f]) / S.sdx[f] : 0.0f;
#pragma unroll
            for (int j = 0; j < TC_KIN / 8; j++) {
                __align__(16) bf16 h[8];
#pragma unroll
                for (int e = 0; e < 8; e++) h[e] = __float2bfloat16_rn(x[8 * j + e]);
                *reinterpret_cast<uint4 *>(Ab + core_off(t, 8 * j, TC_KIN)) = *reinterpret_cast<const uint4 *>(h);
            }
        }
        for (int l = 0; l < 4 && ok; l++) {
            const int K = l == 0 ? TC_KIN : TC_NH, N = l == 3 ? TC_NO : TC_NH;
            // the operand written by every thread, visible to the tensor cores
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t id = idesc_bf16(TC_T, N);
                for (int kk = 0; kk < K / 16; kk++)
                    mma_issue(tmem, sdesc(sA + kk * 256, 128, 16 * K), sdesc(sW[l] + kk * 256, 128, 16 * K), id,
                              kk > 0 ? 1u : 0u);
                mma_commit(bar);
            }
            // the same outcome in every thread, so that all leave together
            ok = __syncthreads_and(bar_wait(bar, phase) ? 1 : 0) != 0;
            if (!ok) break;
            phase ^= 1u;
            fence_after();
            if (l < 3) {
                // bias, tanh, BF16: the next layer's operand (K = 128), in place
#pragma unroll 1
                for (int c1 = 0; c1 < TC_NH; c1 += 64) {
                    // four loads of 16 columns in flight, one wait
                    uint32_t acc[4][16];
                    __syncwarp();
#pragma unroll
                    for (int g = 0; g < 4; g++) tmem_ld16_issue(lane_addr + (uint32_t)(c1 + 16 * g), acc[g]);
#pragma unroll
                    for (int g = 0; g < 4; g++) tmem_ld_wait(acc[g]);
#pragma unroll
                    for (int g = 0; g < 4; g++) {
                        const int c0 = c1 + 16 * g;
                        __align__(16) bf16 h[16];
#pragma unroll
                        for (int e = 0; e < 16; e++)
                            h[e] = __float2bfloat16_rn(tanh_sfu(__uint_as_float(acc[g][e]) + S.b[l][c0 + e]));
                        *reinterpret_cast<uint4 *>(Ab + core_off(t, c0, TC_NH)) = *reinterpret_cast<const uint4 *>(h);
                        *reinterpret_cast<uint4 *>(Ab + core_off(t, c0 + 8, TC_NH)) =
                            *reinterpret_cast<const uint4 *>(h + 8);
                    }
                }
                fence_before();
            } else {
                float v[16];
                tmem_ld16(lane_addr, v);
                if (row < a.n)
#pragma unroll
                    for (int o = 0; o < 4; o++) a.Y[row * 4 + o] = S.muy[o] + S.sdy[o] * (v[o] + S.b3[o]);
                fence_before();
            }
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(a.err, 1);
        if (weights_ok) bar_wait(bar, phase);   // the chain in flight, if it still completes
        else bar_wait(wbar, 0u);                // the copies in flight, if they still complete
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_COLS));
}

}  // namespace

size_t mlp_tc_smem() { return sizeof(TcSmem); }

cudaError_t mlp_tc_prepare()
{
    return cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
}

cudaError_t launch_mlp_forward_tc(const TcArgs &a, int sm_count, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const int ntiles = (int)((a.n + TC_T - 1) / TC_T);
    const int grid = ntiles < sm_count ? ntiles : sm_count;
    k_mlp_forward_tc<<<grid, TC_T, sizeof(TcSmem), st>>>(a);
    return cudaGetLastError();
}

}  // namespace msd
