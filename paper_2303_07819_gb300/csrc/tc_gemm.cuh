// tc_gemm.cuh -- one 128 x 64 tile of C = A B^T on the tcgen05 tensor cores,
// BF16 operands, FP32 accumulation in tensor memory.
//
// A is [M][lda] and B is [N][ldb], both row-major BF16 with K contiguous
// (lda, ldb and the k range multiples of 8, rows 16-byte aligned).  A CTA of
// 128 threads takes rows m0 .. m0 + 127 of C and columns n0 .. n0 + 63 over
// the k range [kbeg, kend).  The threads stage 64-wide k chunks of A and B
// into shared memory in the core-matrix layout, two buffers deep, and one
// thread issues one tcgen05.mma (K = 16) per 16 k of the chunk into a
// 64-column accumulator; a chunk's commit to its buffer's mbarrier frees that
// buffer, so staging chunk c + 1 overlaps the MMAs of chunk c.  Rows of A
// past M, rows of B past N and k past kend read as zero; row `ones_row` of B
// (if >= 0) reads as 1 everywhere, which appends the row sums of A over k to
// C as its column ones_row.
//
// Row i of the accumulator is tensor-memory lane i: after tcg_mainloop
// returns true, thread t of the CTA reads row m0 + t with tcgen05.ld at
// column offsets 0 .. Np - 1 of tmem + (warp * 32 << 16).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "tc_ptx.cuh"

namespace msd {
namespace tcx {

constexpr int TCG_T = 128, TCG_BK = 64, TCG_NT = 64;

struct TcgSmem {
    __nv_bfloat16 A[2][TCG_T * TCG_BK];    // 128 x 64 per buffer, core-matrix layout
    __nv_bfloat16 B[2][TCG_NT * TCG_BK];   // 64 x 64
    unsigned long long bar[2];             // MMA chunk done, per buffer
    uint32_t tbase;
};

// per buffer: the phase of its next commit and whether one is unwaited
struct TcgState {
    uint32_t ph0 = 0u, ph1 = 0u;
    bool pend0 = false, pend1 = false;
};

// barriers and the tensor-memory columns; every thread of the CTA calls it
__device__ __forceinline__ uint32_t tcg_init(TcgSmem &S)
{
    const int t = threadIdx.x;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&S.bar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&S.bar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((t >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S.tbase)), "r"(TCG_NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    return S.tbase;
}

// The tile's MMAs; true when the accumulator holds the tile (false if a wait
// ran out: the same outcome in every thread).  Every thread calls it.
__device__ __forceinline__ bool tcg_mainloop(TcgSmem &S, uint32_t tmem, TcgState &st, int M, int N, int kbeg, int kend,
                                             int m0, int n0, const __nv_bfloat16 *__restrict__ A, int lda,
                                             const __nv_bfloat16 *__restrict__ B, int ldb, int ones_row)
{
    const int t = threadIdx.x;
    const int nch = kend > kbeg ? (kend - kbeg + TCG_BK - 1) / TCG_BK : 0;
    const int Nt = min(TCG_NT, N - n0), Np = (Nt + 15) / 16 * 16;
    const uint32_t bar0 = smem_u32(&S.bar[0]), bar1 = smem_u32(&S.bar[1]);
    for (int c = 0; c < nch; c++) {
        const int b = c & 1, k0 = kbeg + c * TCG_BK;
        const uint32_t bar = b ? bar1 : bar0;
        if (b ? st.pend1 : st.pend0) {
            // buffer b is free once chunk c - 2's MMAs are done
            if (__syncthreads_and(bar_wait(bar, b ? st.ph1 : st.ph0) ? 1 : 0) == 0) return false;
            if (b) { st.ph1 ^= 1u; st.pend1 = false; } else { st.ph0 ^= 1u; st.pend0 = false; }
            fence_after();
        }
        unsigned char *Ab = reinterpret_cast<unsigned char *>(S.A[b]), *Bb = reinterpret_cast<unsigned char *>(S.B[b]);
        // 16-byte pieces, all loads first
        constexpr int PA = TCG_T * (TCG_BK / 8) / TCG_T, PB = TCG_NT * (TCG_BK / 8) / TCG_T;
        uint4 va[PA], vb[PB];
#pragma unroll
        for (int i = 0; i < PA; i++) {
            const int q = t + i * TCG_T, r = q / (TCG_BK / 8), gk = k0 + 8 * (q % (TCG_BK / 8));
            va[i] = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M && gk < kend) va[i] = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + gk);
        }
#pragma unroll
        for (int i = 0; i < PB; i++) {
            const int q = t + i * TCG_T, r = q / (TCG_BK / 8), gk = k0 + 8 * (q % (TCG_BK / 8));
            vb[i] = make_uint4(0u, 0u, 0u, 0u);
            if (r < Nt && gk < kend) {
                if (n0 + r == ones_row) vb[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
                else vb[i] = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + gk);
            }
        }
#pragma unroll
        for (int i = 0; i < PA; i++) {
            const int q = t + i * TCG_T;
            *reinterpret_cast<uint4 *>(Ab + core_off(q / (TCG_BK / 8), 8 * (q % (TCG_BK / 8)), TCG_BK)) = va[i];
        }
#pragma unroll
        for (int i = 0; i < PB; i++) {
            const int q = t + i * TCG_T;
            *reinterpret_cast<uint4 *>(Bb + core_off(q / (TCG_BK / 8), 8 * (q % (TCG_BK / 8)), TCG_BK)) = vb[i];
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (t == 0) {
            const uint32_t id = idesc_bf16(TCG_T, Np), sA = smem_u32(S.A[b]), sB = smem_u32(S.B[b]);
            const int nk = min(TCG_BK / 16, (kend - k0 + 15) / 16);   // k past the range is zero
            for (int kk = 0; kk < nk; kk++)
                mma_issue(tmem, sdesc(sA + kk * 256, 128, 16 * TCG_BK), sdesc(sB + kk * 256, 128, 16 * TCG_BK), id,
                          (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar);
        }
        if (b) st.pend1 = true; else st.pend0 = true;
    }
    if (nch == 0) return true;
    // the last chunk's commit covers every MMA before it
    const int b = (nch - 1) & 1;
    if (__syncthreads_and(bar_wait(b ? bar1 : bar0, b ? st.ph1 : st.ph0) ? 1 : 0) == 0) return false;
    if (b) st.ph1 ^= 1u; else st.ph0 ^= 1u;
    st.pend0 = st.pend1 = false;
    fence_after();
    return true;
}

// After a wait ran out: report it and wait (bounded) for the MMAs in flight
// (at most one commit per buffer).  Then, in every case, free the columns.
__device__ __forceinline__ void tcg_finish(TcgSmem &S, uint32_t tmem, const TcgState &st, bool ok, int *err)
{
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(err, 1);
        if (st.pend0) bar_wait(smem_u32(&S.bar[0]), st.ph0);
        if (st.pend1) bar_wait(smem_u32(&S.bar[1]), st.ph1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCG_NT));
}

}  // namespace tcx
}  // namespace msd
