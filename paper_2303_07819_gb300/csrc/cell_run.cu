// cell_run.cu -- FP32 msDEM cell steps for a whole run of fine steps in one
// launch, every floe resident in a thread's registers (launch variant 5).
//
// Between two coarse steps a cell depends on nothing but itself (Sec. 3.1:
// each coarse cell carries its own doubly periodic DEM; the gradual-update
// increments of Algorithm 1 are fixed at the coarse step), so a block can
// take its cells through every fine step of a run and touch global memory
// only at the run's two ends.
//
// Work: the cells are packed into groups of at most 256 K floes (K = 1, 2
// or 4 floes per thread of a 256-thread block): a cell of more than 256
// (K = 2) or 512 (K = 4) floes is a group of its own, smaller cells share
// K = 1 groups, first fit by decreasing size.  A cell's floes so always run
// the code of its own size class, whatever else the model holds.  Each K is one persistent
// launch whose blocks take groups from a ticket queue in decreasing order of
// work.  A floe's state, forcing and running sums stay in registers for the
// run; per step it publishes its position and velocity to shared memory (two
// buffers, so one barrier per step separates the step that reads a buffer
// from the one that writes it again).
//
// Contacts (Eq. 2.2): a floe tests only its candidates, the floes of its
// cell within reach at the last build: r_l G + s_l + r_j G + s_j, with G the
// growth the cell's gradual updates can still give its radii in this
// coarse interval and s_f the floe's own skin (its speed times a horizon of
// steps).  A build is a counting sort of the group's floes into per-cell
// bins (floes whose reach fits half a bin) and a per-cell list of the other,
// "large" floes; small floes search their 3 x 3 bins and the large list
// (recording a hit on both sides), large floes the large list.  A group
// builds at the first step of a run and again once a floe has moved more
// than its skin.  A list holds at most LMAX candidates; a floe whose list
// overflowed tests every floe of its cell instead.  Each list is sorted by
// floe index, so a floe always sums its contacts in ascending partner order
// -- the order of the all-pairs loop over (l < j) in cell order, whatever
// the skins, bins or build steps were.
//
// Ocean (Eq. 2.1c-d at the floe's global position): each floe keeps the
// first-order Taylor expansion of the current and its curl about a centre
// near it and evaluates that every step (6 multiply-adds instead of a sum
// of modes).  The neglected term stays below the FP32 rounding of the mode
// sum while the floe is within sqrt(P.ocean_d2) of the centre (the bound is
// derived from the modes' wave numbers on the host); when a floe of a cell
// goes farther, or wraps across its cell's edge, every floe of that cell
// expands again at its current position with the modes' full sums at the
// next step (a decision of the cell alone, whichever cells share its block).
//
// Moments (Algorithm 1): the window needs per step the cell's mass-weighted
// mean velocity and its drag totals.  A gradual update scales the radii of
// all floes of a cell by one factor (Eq. 3.5 with reading c11) and leaves
// thicknesses alone, so each floe's share m_f / M of its cell's mass is the
// same at every step of a coarse interval; then sum_s (sum_f m_f u_f,s) / M
// = sum_f (m_f / M) (sum_s u_f,s).  Each floe sums its velocity and drag
// over the interval and the block reduces these sums once, at the
// interval's end.  A run that ends inside an interval stores the floes'
// running sums and expansion centres (the carry) and the next run picks
// them up, so a coarse interval gives the same result bit for bit however
// it is split into runs.  The cell moments of the run's
// last step (all 12 columns) are reduced once at the end.  Reductions are
// segmented warp shuffles in a fixed tree, then a cell's warp partials in
// order in FP64: deterministic.
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "common.cuh"
#include "fixsum.cuh"

namespace msd {

namespace {

// Tunables (measured on the 128 x 128 batched workload; see the build flags)
#ifndef MS_RUN_LMAX
#define MS_RUN_LMAX 16
#endif
#ifndef MS_RUN_K1_BLOCKS
#define MS_RUN_K1_BLOCKS 4
#endif
#ifndef MS_RUN_K2_BLOCKS
#define MS_RUN_K2_BLOCKS 2
#endif

constexpr int RT = RUN_T;          // threads per block
constexpr int LMAX = MS_RUN_LMAX;  // candidate slots per floe
constexpr int GCMAX = RUN_GCMAX;   // cells per group
constexpr int WT = 128;            // steps per wind table
constexpr int NRED = 16;           // values per reduction (moment columns 1-11, window sums)
constexpr int NEVT = 32;           // gradual updates per interval with a precomputed radius ratio

template <int K>
struct RunSm {
    static constexpr int F = RT * K;
    uint2 Q[2][F];                  // fixed-point position, per step buffer
    float4 A[2][F];                 // u, v, w, r
    float H[F];                     // thickness
    float RE[F];                    // reach of each floe at the build: r G + s
    unsigned short L[LMAX][F];      // candidate lists, slot-major (conflict-free by floe)
    int LC[F];                      // list lengths (other floes append during a build)
    unsigned short SF[F];           // floes in bin order (build)
    unsigned short BF[F];           // bin of each floe (build)
    int BS[F + GCMAX + 1];          // bin counts, then starts
    int BC[F + GCMAX + 1];          // bin cursors
    unsigned long long csum[NRED][GCMAX];   // per-cell sums of a reduction, fixed point (two's complement)
    int cexp[NRED][GCMAX];          // their binary exponents: the largest of the cell's values
    float2 Cm[GCMAX][MAXM];         // per cell and mode: corner phase (cos, sin), or (cycles, -)
    float rg[2][GCMAX][4];          // gradual update per cell (g, du, dv, dw), by step parity
    float cgrow[GCMAX][NEVT + 1];   // growth the cell's radii can still take this interval, by updates done
    float cdv[GCMAX][NEVT + 1];     // speed the cell's gradual updates can still add, by updates done
    double cwin[GCMAX][NWIN];       // the cells' window sums (loaded at the run's start, stored at its end)
    float rgev[GCMAX][NEVT];        // radius ratio of each gradual update of the interval, per cell
    float2 wind[WT];
    int cc[GCMAX], cfs[GCMAX], cn[GCMAX], cnb[GCMAX], cbb[GCMAX], cgo[GCMAX];
    int cskip[GCMAX];               // a closure cell: no DEM this interval (its floes stay where they are)
    int ncg, nfl, nbin, item, allskip;
    float vsum[2];                  // group speed sums of the builds, by build parity
    int cflag[3][GCMAX];            // a floe of the cell strayed from its ocean centre, by step mod 3
};

__host__ __device__ constexpr size_t run_smem_bytes(int K)
{
    return K == 1 ? sizeof(RunSm<1>) : (K == 2 ? sizeof(RunSm<2>) : sizeof(RunSm<4>));
}

// Segmented warp reductions towards the head of each segment: lanes [lane,
// end) of this warp belong to the caller's segment; after the call the
// segment's first lane holds its maximum or total.  Integer operations, so
// the result does not depend on the order.
__device__ __forceinline__ int seg_max(int x, int lane, int end_lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_down_sync(0xffffffffu, x, d);
        if (lane + d < end_lane) x = max(x, y);
    }
    return x;
}

__device__ __forceinline__ long long seg_sum(long long x, int lane, int end_lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_down_sync(0xffffffffu, x, d);
        if (lane + d < end_lane) x += y;
    }
    return x;
}

// Exclusive scan of BS[0..nb) in place (block-wide); BC gets a copy of the
// starts.  Ends with a barrier.
template <int K>
__device__ void block_scan_bins(RunSm<K> &S, int nb)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = RT / 32;
    __shared__ int wsum[NW];
    const int per = (nb + RT - 1) / RT;
    const int b0 = t * per, b1 = min(b0 + per, nb);
    int s = 0;
    for (int b = b0; b < b1; b++) s += S.BS[b];
    int x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int wbase = 0;
    for (int k = 0; k < warp; k++) wbase += wsum[k];
    int run = wbase + x - s;
    for (int b = b0; b < b1; b++) {
        const int c = S.BS[b];
        S.BS[b] = run;
        S.BC[b] = run;
        run += c;
    }
    __syncthreads();
}

// |(a, b)| from the hardware reciprocal square root (within a few ulp of
// the correctly rounded norm; 0 for the zero vector)
__device__ __forceinline__ float fast_norm(float a, float b)
{
    const float q = fmaf(a, a, b * b);
    return q > 0.0f ? q * rsqrtf(q) : 0.0f;
}

// Has a floe at fixed point (xq, yq) left the region where the first-order
// expansion of the current about (x0, y0) holds (squared distance above d2),
// or wrapped across its cell's edge since (its global position jumped by a
// cell side while the fixed-point difference stayed small)?
__device__ __forceinline__ bool ocean_stale(uint32_t xq, uint32_t yq, uint32_t x0, uint32_t y0, float sx, float sy,
                                            float d2)
{
    const int ix = (int)(xq - x0), iy = (int)(yq - y0);
    const float dx = (float)ix * sx, dy = (float)iy * sy;
    const bool wrapped = (xq < x0) != (ix < 0) || (yq < y0) != (iy < 0);
    return wrapped || dx * dx + dy * dy > d2;
}

// Ocean current and curl, and their gradients (per metre of global X, Y),
// at the fraction (xf, yf) of cell ci: the modes' full sums in the FP32
// phase-split form (corner phase Cm, turn across the cell).
struct OceanExp {
    float u, v, z, ux, uy, vx, vy, zx, zy;
};

template <int K>
__device__ __forceinline__ OceanExp ocean_expand(const Phys<float> &P, const RunSm<K> &S, int ci, float xf, float yf,
                                                 float inx, float iny)
{
    OceanExp o;
    o.u = P.uo_x; o.v = P.uo_y; o.z = 0.0f;
    o.ux = o.uy = o.vx = o.vy = o.zx = o.zy = 0.0f;
    for (int m = 0; m < P.n_modes; m++) {
        float cs, sn;
        if (P.taylor) {
            float c0, s0;
            rot_small(fmaf(P.ta[m], xf, P.tb[m] * yf), c0, s0);
            const float2 C = S.Cm[ci][m];
            cs = C.x * c0 - C.y * s0;
            sn = C.y * c0 + C.x * s0;
        } else {
            const float cyc = S.Cm[ci][m].x + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
            sincospif(2.0f * cyc, &sn, &cs);
        }
        // mode m: u -= Au cos(th), v += Av cos(th), curl -= Az sin(th), th = kx X + ky Y + phi
        const float kx = P.mKx[m], ky = P.mKy[m];
        const float au = P.mAu[m], av = P.mAv[m], az = P.mAz[m];
        o.u -= au * cs;
        o.v += av * cs;
        o.z -= az * sn;
        const float aus = au * sn, avs = av * sn, azc = az * cs;
        o.ux += aus * kx;
        o.uy += aus * ky;
        o.vx -= avs * kx;
        o.vy -= avs * ky;
        o.zx -= azc * kx;
        o.zy -= azc * ky;
    }
    return o;
}

template <int K>
__global__ void __launch_bounds__(RT, K == 1 ? MS_RUN_K1_BLOCKS : (K == 2 ? MS_RUN_K2_BLOCKS : 1))
k_cell_run32_block(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, const int4 *groups, int ngroups,
                   const int4 *items, int qslot, int nsteps, float skin_steps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RunSm<K> &S = *reinterpret_cast<RunSm<K> *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31;
    const unsigned FULL = 0xffffffffu;
    const float dt = sc.k.dt;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy;
    const float Lcmin = fminf(sc.k.Lx, sc.k.Ly);
    const int nc = sc.ncell;
    const long long base = sc.ctrl->base;
    const int j0 = (int)sc.i_local;                     // steps of the interval done before this run
    const bool have_tgt = sc.couple && sc.ctrl->have_tgt;
    const bool win_on = sc.couple != 0;
    const bool ends_interval = sc.couple && (j0 + nsteps == sc.N0);
    const bool carry_in = win_on && j0 > 0;             // the run continues a previous one inside its interval
    const bool carry_out = win_on && !ends_interval;
    const float dtsx = dt * isx, dtsy = dt * isy;
    const long long ncar = sc.ncarry;
    const int nev = sc.N0 / sc.n_t;                     // gradual updates per interval

    // wind of steps [js0, js0 + WT) of the run (FP64 turn, once per block
    // for runs of up to WT steps)
    auto wind_table = [&](int js0) {
        if (t < WT && js0 + t < nsteps) {
            float ua, va;
            wind_at(P, (double)(base + j0 + js0 + t) * sc.dt, ua, va);
            S.wind[t] = make_float2(ua, va);
        }
    };
    wind_table(0);

    for (;;) {
        // ---- next group from the queue
        __syncthreads();
        if (t == 0) {
            int g = (int)atomicAdd(&sc.ctrl->gq[qslot][0], 1u);
            if (g >= ngroups) {
                __threadfence();
                const unsigned done = atomicAdd(&sc.ctrl->gq[qslot][1], 1u);
                if (done == gridDim.x - 1) {     // the last block out resets the queue for the next launch
                    sc.ctrl->gq[qslot][0] = 0u;
                    sc.ctrl->gq[qslot][1] = 0u;
                    __threadfence();
                }
            }
            S.item = g;
        }
        __syncthreads();
        const int gid = S.item;
        if (gid >= ngroups) return;

        // ---- the group's cells
        const int4 gd = groups[gid];          // first slot, cells, floes, bins (with one large slot per cell)
        if (t < 32) {                         // warp 0: a group has at most 32 cells
            int n = 0;
            if (t < gd.y) {
                const int4 id = items[gd.x + t];  // cell, first floe in the group, bins per side, bin base
                const int c = id.x;
                const int skip = sc.skip && sc.skip[c] ? 1 : 0;
                n = skip ? 0 : sc.off[c + 1] - sc.off[c];
                S.cc[t] = c;
                S.cskip[t] = skip;
                S.cn[t] = n;
                S.cnb[t] = id.z;
                S.cbb[t] = id.w;
                S.cgo[t] = sc.off[c];
            }
            // the group's floes packed cell after cell, closure cells holding
            // none (without a closure: the places the grouping gave them)
            int x = n;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(FULL, x, d);
                if (lane >= d) x += y;
            }
            if (t < gd.y) S.cfs[t] = x - n;
            if (t == 31) S.nfl = x;
            const unsigned sk = __ballot_sync(FULL, t < gd.y && sc.skip && sc.skip[S.cc[t]]);
            if (t == 0) S.allskip = __popc(sk) == gd.y;
        }
        if (t == 0) {
            S.ncg = gd.y;
            S.nbin = gd.w;
        }
        if (t < 3 * GCMAX) (&S.cflag[0][0])[t] = 0;
        __syncthreads();
        if (S.allskip) continue;              // every cell of the group takes the closure this interval
        const int ncg = S.ncg, nfl = S.nfl;
        for (int idx = t; idx < ncg * P.n_modes; idx += RT) {
            const int ci = idx / P.n_modes, m = idx - ci * P.n_modes;
            const int c = S.cc[ci];
            const float b = corner_phase(P, m, c % sc.g.nx, (c / sc.g.nx) % sc.g.nyr, sc.g.nx, sc.g.nyr, sc.k.inx,
                                         sc.k.iny);
            if (P.taylor) {
                float sn, cs;
                sincospif(2.0f * b, &sn, &cs);
                S.Cm[ci][m] = make_float2(cs, sn);
            } else {
                S.Cm[ci][m] = make_float2(b, 0.0f);
            }
        }
        // the window sums so far, added to in sequence and stored at the run's
        // end (the same additions however the interval is split into runs)
        if (t < ncg)
            for (int q = 0; q < NWIN; q++) S.cwin[t][q] = win_on ? sc.win[(size_t)q * nc + S.cc[t]] : 0.0;
        // per cell and gradual update of the interval (FP64, once): the
        // update's radius ratio; and, by the updates already applied, the
        // growth the radii can still take (r goes to r0 s at the last update
        // from r0 (1 + (s - 1) ev n_t/N0) after update ev) and the velocity the
        // remaining updates add (n_t/N0 of the target each)
        const int nevt = have_tgt && nev <= NEVT ? nev : 0;
        for (int idx = t; idx < ncg * (nevt + 1); idx += RT) {
            const int ci = idx / (nevt + 1), ev = idx - ci * (nevt + 1);
            const int c = S.cc[ci];
            const double s = sc.tgt[c];
            if (ev >= 1) S.rgev[ci][ev - 1] = (float)ramp_cell(sc, c, ev).g;
            float gr = 1.0f, dvr = 0.0f;
            if (nevt) {
                const double g = s / (1.0 + (s - 1.0) * ev / (double)nev);
                gr = g > 1.0 ? (float)(g * (1.0 + 1e-6)) : 1.0f;
                const double du = sc.tgt[nc + c], dv = sc.tgt[2 * nc + c];
                dvr = (float)(sqrt(du * du + dv * dv) * (nev - ev) / (double)nev);
            }
            S.cgrow[ci][ev] = gr;
            S.cdv[ci][ev] = dvr;
        }
        if (t == 0) S.vsum[0] = S.vsum[1] = 0.0f;
        int nbuild = 0;
        // gradual update of the run's first step, if it is one
        if (t < ncg) {
            const int kk = j0 + 1;
            float g = 1.0f, du = 0.0f, dv = 0.0f, dw = 0.0f;
            if (have_tgt && kk % sc.n_t == 0) {
                const RampCell rc = ramp_cell(sc, S.cc[t], kk / sc.n_t);
                g = (float)rc.g; du = (float)rc.du; dv = (float)rc.dv; dw = (float)rc.dw;
            }
            S.rg[0][t][0] = g; S.rg[0][t][1] = du; S.rg[0][t][2] = dv; S.rg[0][t][3] = dw;
        }

        // ---- this thread's floes: p = t + k RT in group order
        int ci[K], lc[K];
        uint32_t xq[K], yq[K], xb[K], yb[K], x0[K], y0[K];
        float th[K], u[K], v[K], w[K], r[K], h[K], dtm[K], dtI[K], sk2[K];
        float su[K], sv[K], sfx[K], sfy[K], stz[K];
        OceanExp oc[K];
        unsigned deep = 0;
        bool bad = false;
        auto derived = [&](int k) {
            const float mass = P.mass_c * r[k] * r[k] * h[k];
            const float I = P.inertia_f * mass * r[k] * r[k];
            dtm[k] = dt / mass;
            dtI[k] = dt / I;
        };
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int p = t + k * RT;
            ci[k] = 0;
            lc[k] = 0;
            xq[k] = yq[k] = xb[k] = yb[k] = 0u;
            th[k] = u[k] = v[k] = w[k] = 0.0f;
            r[k] = 1.0f;
            h[k] = 1.0f;
            sk2[k] = 0.0f;
            su[k] = sv[k] = sfx[k] = sfy[k] = stz[k] = 0.0f;
            if (p < nfl) {
                int c2 = 0;
                while (c2 + 1 < ncg && S.cfs[c2 + 1] <= p) c2++;
                ci[k] = c2;
                const int gi = S.cgo[c2] + (p - S.cfs[c2]);
                xq[k] = in.xq[gi]; yq[k] = in.yq[gi]; th[k] = in.th[gi];
                u[k] = in.u[gi]; v[k] = in.v[gi]; w[k] = in.w[gi]; r[k] = in.r[gi]; h[k] = in.h[gi];
                S.Q[0][p] = make_uint2(xq[k], yq[k]);
                S.A[0][p] = make_float4(u[k], v[k], w[k], r[k]);
                S.H[p] = h[k];
            }
            x0[k] = xq[k];
            y0[k] = yq[k];
            if (carry_in && p < nfl) {
                const int gi = S.cgo[ci[k]] + (p - S.cfs[ci[k]]);
                su[k] = sc.carry_in[gi];
                sv[k] = sc.carry_in[ncar + gi];
                sfx[k] = sc.carry_in[2 * ncar + gi];
                sfy[k] = sc.carry_in[3 * ncar + gi];
                stz[k] = sc.carry_in[4 * ncar + gi];
                x0[k] = __float_as_uint(sc.carry_in[5 * ncar + gi]);
                y0[k] = __float_as_uint(sc.carry_in[6 * ncar + gi]);
            }
            derived(k);
        }
        // the ocean expansions are made in the step loop (one call site, so
        // every expansion rounds alike): at the first step about the centres
        // above, later whenever a floe of the warp strays
        bool expand_at_centre = true;

        // ---- reduction of NV (<= NRED) per-floe values per cell, exact and
        // independent of where the cell's floes sit in the block: the
        // largest binary exponent of each (cell, column), then the values in
        // fixed point relative to it summed as integers (segments of a warp
        // by shuffles, their heads into shared memory atomically); head_sum
        // converts a total back.  All threads call seg_partials; it begins
        // and ends with a barrier.
        auto seg_partials = [&](auto nv, auto &&value) {
            constexpr int NV = decltype(nv)::value;
            for (int i = t; i < NV * GCMAX; i += RT) {
                S.cexp[i / GCMAX][i % GCMAX] = FIX_NONE;
                S.csum[i / GCMAX][i % GCMAX] = 0ull;
            }
            __syncthreads();
            // a value counts if it is finite and nonzero (a non-finite state
            // is reported by the run's end check)
            auto counted = [&](int k, int q, bool valid) -> float {
                return fix_counted(valid ? value(k, q) : 0.0f);
            };
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                const bool valid = p < nfl;
                const int fs = valid ? S.cfs[ci[k]] : nfl;
                const int fe = valid ? S.cfs[ci[k]] + S.cn[ci[k]] : RT * K;
                const int wb = p & ~31;
                const int end_lane = min(fe, wb + 32) - wb;
                const int head = max(fs, wb);
#pragma unroll
                for (int q = 0; q < NV; q++) {
                    const float x = counted(k, q, valid);
                    const int e = seg_max(fix_exp(x), lane, end_lane);
                    if (p == head && e != FIX_NONE) atomicMax(&S.cexp[q][ci[k]], e);
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                const bool valid = p < nfl;
                const int fs = valid ? S.cfs[ci[k]] : nfl;
                const int fe = valid ? S.cfs[ci[k]] + S.cn[ci[k]] : RT * K;
                const int wb = p & ~31;
                const int end_lane = min(fe, wb + 32) - wb;
                const int head = max(fs, wb);
#pragma unroll
                for (int q = 0; q < NV; q++) {
                    const float x = counted(k, q, valid);
                    const long long iv = seg_sum(fix_val(x, S.cexp[q][ci[k]]), lane, end_lane);
                    if (p == head && iv != 0) atomicAdd(&S.csum[q][ci[k]], (unsigned long long)iv);
                }
            }
            __syncthreads();
        };
        auto head_sum = [&](int cell, int q) -> double {
            return fix_total((long long)S.csum[q][cell], S.cexp[q][cell]);
        };
        // ---- candidate lists from the positions in buffer b, before step kk
        auto build = [&](int b, int kk) {
            // the floor of the skins: a quarter of the group's mean speed
            float vs = 0.0f;
#pragma unroll
            for (int k = 0; k < K; k++)
                if (t + k * RT < nfl) vs += sqrtf(u[k] * u[k] + v[k] * v[k]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) vs += __shfl_xor_sync(FULL, vs, d);
            for (int i = t; i <= S.nbin; i += RT) S.BS[i] = 0;
            if (have_tgt && !nevt && t < ncg) {   // more updates per interval than the table holds
                const int c = S.cc[t];
                const double s = sc.tgt[c];
                const int ev = (kk - 1) / sc.n_t;
                const double g = s / (1.0 + (s - 1.0) * ev / (double)nev);
                const double du = sc.tgt[nc + c], dv = sc.tgt[2 * nc + c];
                S.cgrow[t][0] = g > 1.0 ? (float)(g * (1.0 + 1e-6)) : 1.0f;
                S.cdv[t][0] = (float)(sqrt(du * du + dv * dv) * (nev - ev) / (double)nev);
            }
            const int vb = nbuild & 1;
            if (lane == 0) atomicAdd(&S.vsum[vb], vs);
            if (t == 0) S.vsum[vb ^ 1] = 0.0f;    // for the next build
            __syncthreads();
            // updates already applied (radius growth and velocity still to come)
            int evd = (kk - 1) / sc.n_t;
            if (!nevt) evd = 0;
            const float vfloor = 0.25f * S.vsum[vb] / (float)max(nfl, 1);
            nbuild++;
            const float horizon = skin_steps * dt;
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                if (p < nfl) {
                    const int c2 = ci[k], nb = S.cnb[c2];
                    const float sp = sqrtf(u[k] * u[k] + v[k] * v[k]) + S.cdv[c2][evd];
                    const float skin = (1.5f * sp + vfloor) * horizon + 1.0e-3f * r[k];
                    sk2[k] = skin * skin;
                    const float reach = r[k] * S.cgrow[c2][evd] + skin;
                    S.RE[p] = reach;
                    const bool small = nb >= 3 && reach <= 0.5f * (Lcmin / (float)nb);
                    const int bn = S.cbb[c2] + (small ? (int)(__umulhi(yq[k], (unsigned)nb) * nb +
                                                               __umulhi(xq[k], (unsigned)nb))
                                                      : nb * nb);
                    S.BF[p] = (unsigned short)bn;
                    atomicAdd(&S.BS[bn], 1);
                    S.LC[p] = 0;
                }
            }
            __syncthreads();
            block_scan_bins(S, S.nbin + 1);   // BS[nbin] = the group's floes
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                if (p < nfl) S.SF[atomicAdd(&S.BC[S.BF[p]], 1)] = (unsigned short)p;
            }
            __syncthreads();
            // search
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                if (p >= nfl) continue;
                const int c2 = ci[k], nb = S.cnb[c2], bb = S.cbb[c2];
                const uint2 ql = make_uint2(xq[k], yq[k]);
                const float rl = S.RE[p];
                auto hit = [&](int q) {
                    const uint2 qq = S.Q[b][q];
                    const float dx = (float)(int)(qq.x - ql.x) * sx, dy = (float)(int)(qq.y - ql.y) * sy;
                    const float Ssum = rl + S.RE[q];
                    return fmaf(Ssum, Ssum, -(dx * dx + dy * dy)) > 0.0f;
                };
                auto add = [&](int a, int q) {
                    const int slot = atomicAdd(&S.LC[a], 1);
                    if (slot < LMAX) S.L[slot][a] = (unsigned short)q;
                };
                const int lg0 = S.BS[bb + nb * nb], lg1 = S.BS[bb + nb * nb + 1];   // the cell's large floes
                const bool small = (int)S.BF[p] != bb + nb * nb;
                if (small) {
                    const int bx = (int)__umulhi(ql.x, (unsigned)nb), by = (int)__umulhi(ql.y, (unsigned)nb);
                    for (int dyb = -1; dyb <= 1; dyb++) {
                        int wy = by + dyb;
                        wy = wy < 0 ? wy + nb : (wy >= nb ? wy - nb : wy);
                        const int row = bb + wy * nb;
                        for (int dxb = -1; dxb <= 1; dxb++) {
                            int wx = bx + dxb;
                            wx = wx < 0 ? wx + nb : (wx >= nb ? wx - nb : wx);
                            const int e1 = S.BS[row + wx + 1];
                            for (int i = S.BS[row + wx]; i < e1; i++) {
                                const int q = S.SF[i];
                                if (q != p && hit(q)) add(p, q);
                            }
                        }
                    }
                    for (int i = lg0; i < lg1; i++) {     // small-large pairs: both sides recorded here
                        const int q = S.SF[i];
                        if (hit(q)) {
                            add(p, q);
                            add(q, p);
                        }
                    }
                } else {
                    for (int i = lg0; i < lg1; i++) {     // large-large pairs: each side its own
                        const int q = S.SF[i];
                        if (q != p && hit(q)) add(p, q);
                    }
                }
            }
            __syncthreads();
            // each list in ascending floe order; the build positions
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int p = t + k * RT;
                if (p >= nfl) continue;
                const int n = S.LC[p];
                lc[k] = n;
                if (n <= LMAX) {
                    for (int i = 1; i < n; i++) {
                        const unsigned short key = S.L[i][p];
                        int j = i - 1;
                        while (j >= 0 && S.L[j][p] > key) {
                            S.L[j + 1][p] = S.L[j][p];
                            j--;
                        }
                        S.L[j + 1][p] = key;
                    }
                }
                xb[k] = xq[k];
                yb[k] = yq[k];
            }
        };

        // the first step's recentring follows the rule of every later step:
        // a cell whose floe strayed from its centre expands again
#pragma unroll
        for (int k = 0; k < K; k++)
            if (t + k * RT < nfl && ocean_stale(xq[k], yq[k], x0[k], y0[k], sx, sy, P.ocean_d2)) S.cflag[0][ci[k]] = 1;
        if (nsteps > WT) wind_table(0);   // a previous group left a later table
        __syncthreads();
        int cur = 0;
        bool need_build = true;
        float Fdl[K][3];                                  // the drag of the latest step (the moments' columns 9-11)
        int ph = (j0 + 1) % sc.n_t;                       // kk mod n_t
        for (int js = 0; js < nsteps; js++) {
            const int kk = j0 + js + 1;                   // step within the interval, 1-based
            if (js > 0 && (js & (WT - 1)) == 0) {
                __syncthreads();
                wind_table(js);
                __syncthreads();
            }
            const bool period_end = ph == 0;
            if (need_build) build(cur, kk);
            __syncthreads();
            const float2 wa = S.wind[js & (WT - 1)];
            const bool ramp = have_tgt && period_end;
            const int rb = js & 1;
            ph = ph + 1 == sc.n_t ? 0 : ph + 1;           // next step's kk mod n_t
            // next step's gradual update, published by the step barrier below
            if (have_tgt && ph == 0 && t < ncg && js + 1 < nsteps) {
                const int ev = (kk + 1) / sc.n_t;
                if (nev <= NEVT) {
                    const double f = (double)sc.n_t / (double)sc.N0;
                    const int c = S.cc[t];
                    S.rg[rb ^ 1][t][0] = S.rgev[t][ev - 1];
                    S.rg[rb ^ 1][t][1] = (float)(sc.tgt[nc + c] * f);
                    S.rg[rb ^ 1][t][2] = (float)(sc.tgt[2 * nc + c] * f);
                    S.rg[rb ^ 1][t][3] = (float)(sc.tgt[3 * nc + c] * f);
                } else {
                    const RampCell rc = ramp_cell(sc, S.cc[t], ev);
                    S.rg[rb ^ 1][t][0] = (float)rc.g;
                    S.rg[rb ^ 1][t][1] = (float)rc.du;
                    S.rg[rb ^ 1][t][2] = (float)rc.dv;
                    S.rg[rb ^ 1][t][3] = (float)rc.dw;
                }
            }
            const bool last = js == nsteps - 1;
            const int fl_cur = js % 3, fl_nxt = (js + 1) % 3;
            if (t < ncg) S.cflag[(js + 2) % 3][t] = 0;     // read two steps ago, written at the next step's end
            bool far = false;
#pragma unroll
            for (int k = 0; k < K; k++) {
                Fdl[k][0] = Fdl[k][1] = Fdl[k][2] = 0.0f;
                const int p = t + k * RT;
                const bool valid = p < nfl;
                // the ocean expansion: every floe of a cell expands again about
                // its current position when one of them strayed at the last
                // step (a decision of the cell alone, whatever shares its
                // block); at the run's first step each floe about its centre
                // unless it strayed from it
                float ex = (float)(int)(xq[k] - x0[k]) * sx, ey = (float)(int)(yq[k] - y0[k]) * sy;
                const bool recentre = valid && S.cflag[fl_cur][ci[k]] != 0;
                if (recentre || expand_at_centre) {
                    if (recentre) {
                        x0[k] = xq[k];
                        y0[k] = yq[k];
                        ex = ey = 0.0f;
                    }
                    oc[k] = ocean_expand(P, S, ci[k], (float)x0[k] * INV2_32F, (float)y0[k] * INV2_32F, sc.k.inx,
                                         sc.k.iny);
                }
                if (!valid) continue;
                // contacts, ascending partner order
                float fx = 0.0f, fy = 0.0f, tq = 0.0f;
                unsigned dflag = 0;
                const uint2 ql = make_uint2(xq[k], yq[k]);
                auto pair = [&](int q) {
                    const uint2 qq = S.Q[cur][q];
                    const float4 aq = S.A[cur][q];
                    const float dx = (float)(int)(qq.x - ql.x) * sx;
                    const float dy = (float)(int)(qq.y - ql.y) * sy;
                    contact_add(dx, dy, dx * dx + dy * dy, r[k], aq.w, h[k], S.H[q], aq.x - u[k], aq.y - v[k], w[k],
                                aq.z, P, fx, fy, tq, dflag);
                };
                // one call site for the pair law: a floe whose list overflowed
                // walks its whole cell in the same order
                const bool brute = lc[k] > LMAX;
                const int cnt = brute ? S.cn[ci[k]] : lc[k], q0 = S.cfs[ci[k]];
                for (int i = 0; i < cnt; i++) {
                    const int q = brute ? q0 + i : (int)S.L[i][p];
                    if (q != p) pair(q);
                }
                deep += dflag;
                // ocean and wind drag (Eq. 2.1c-d)
                const OceanExp &o = oc[k];
                const float uo = fmaf(o.ux, ex, fmaf(o.uy, ey, o.u));
                const float vo = fmaf(o.vx, ex, fmaf(o.vy, ey, o.v));
                const float zeta = fmaf(o.zx, ex, fmaf(o.zy, ey, o.z));
                const float r2 = r[k] * r[k];
                const float ao = P.drag_o * r2, aa = P.drag_a * r2, bo = ao * r2;
                const float du_o = uo - u[k], dv_o = vo - v[k];
                const float so = fast_norm(du_o, dv_o);
                const float au = wa.x - u[k], av = wa.y - v[k];
                const float sa = fast_norm(au, av);
                const float dwo = 0.5f * zeta - w[k];
                const float Fdx = ao * du_o * so + aa * au * sa;
                const float Fdy = ao * dv_o * so + aa * av * sa;
                const float Td = bo * dwo * fabsf(dwo);
                fx += Fdx; fy += Fdy; tq += Td;
                // forward Euler (Sec. 3.1), periodic wrap by fixed-point overflow
                xq[k] += (uint32_t)__float2int_rn(dtsx * u[k]);
                yq[k] += (uint32_t)__float2int_rn(dtsy * v[k]);
                th[k] += dt * w[k];
                u[k] += dtm[k] * fx;
                v[k] += dtm[k] * fy;
                w[k] += dtI[k] * tq;
                if (ramp) {                   // gradual update (Eqs. 3.5-3.7)
                    const float *g4 = S.rg[rb][ci[k]];
                    r[k] *= g4[0];
                    u[k] += g4[1];
                    v[k] += g4[2];
                    w[k] += g4[3];
                    derived(k);
                }
                su[k] += u[k];
                sv[k] += v[k];
                sfx[k] += Fdx;
                sfy[k] += Fdy;
                stz[k] += Td;
                Fdl[k][0] = Fdx; Fdl[k][1] = Fdy; Fdl[k][2] = Td;
                if (!last) {
                    S.Q[cur ^ 1][p] = make_uint2(xq[k], yq[k]);
                    S.A[cur ^ 1][p] = make_float4(u[k], v[k], w[k], r[k]);
                }
                const float bx = (float)(int)(xq[k] - xb[k]) * sx, by = (float)(int)(yq[k] - yb[k]) * sy;
                far |= bx * bx + by * by > sk2[k];
                if (!last && ocean_stale(xq[k], yq[k], x0[k], y0[k], sx, sy, P.ocean_d2)) S.cflag[fl_nxt][ci[k]] = 1;
            }
            need_build = __syncthreads_or(far) != 0;
            expand_at_centre = false;
            cur ^= 1;
        }
        // ---- the run's end: the cell moments of its last step (every column)
        // and, at the interval's end, the window sums of Algorithm 1, in one
        // exact reduction
        {
            auto val = [&](int k, int q) -> float {
                const float m = P.mass_c * r[k] * r[k] * h[k];
                const float I = P.inertia_f * m * r[k] * r[k];
                switch (q) {
                case 0: return m;
                case 1: return m * u[k];
                case 2: return m * v[k];
                case 3: return I;
                case 4: return I * w[k];
                case 5: return 3.14159265358979323846f * r[k] * r[k];
                case 6: return m * u[k] * u[k];
                case 7: return m * v[k] * v[k];
                case 8: return Fdl[k][0];
                case 9: return Fdl[k][1];
                case 10: return Fdl[k][2];
                case 11: return m * su[k];
                case 12: return m * sv[k];
                case 13: return sfx[k];
                case 14: return sfy[k];
                default: return stz[k];
                }
            };
            if (ends_interval) seg_partials(std::integral_constant<int, 16>{}, val);
            else seg_partials(std::integral_constant<int, 11>{}, val);
            // moment columns 1-11 are reduction columns 0-10
            for (int i = t; i < 11 * ncg; i += RT) {
                const int cell = i / 11, q = i - 11 * cell;
                if (!S.cskip[cell]) sc.mom[(size_t)S.cc[cell] * NMOM + 1 + q] = head_sum(cell, q);
            }
            if (t < ncg && !S.cskip[t]) sc.mom[(size_t)S.cc[t] * NMOM] = (double)S.cn[t];
            if (ends_interval) {
                if (t < 5 * ncg) {
                    const int cell = t / 5, q = t - 5 * cell;     // window column
                    const double x = head_sum(cell, 11 + q);
                    if (q < 2) {
                        const double M = head_sum(cell, 0);
                        if (M > 0.0) S.cwin[cell][q] += x / M;
                    } else {
                        S.cwin[cell][q] += x;
                    }
                }
#pragma unroll
                for (int k = 0; k < K; k++) {
                    bad |= !(isfinite(su[k]) && isfinite(sv[k]) && isfinite(stz[k]));
                    su[k] = sv[k] = sfx[k] = sfy[k] = stz[k] = 0.0f;
                }
            }
        }
        __syncthreads();
        if (win_on && t < ncg && !S.cskip[t]) {
            const int c = S.cc[t];
            for (int q = 0; q < NWIN; q++) sc.win[(size_t)q * nc + c] = S.cwin[t][q];
        }
        // ---- back to global memory
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int p = t + k * RT;
            if (p >= nfl) continue;
            bad |= !(isfinite(u[k]) && isfinite(v[k]) && isfinite(w[k]));
            const int gi = S.cgo[ci[k]] + (p - S.cfs[ci[k]]);
            out.xq[gi] = xq[k]; out.yq[gi] = yq[k]; out.th[gi] = th[k];
            out.u[gi] = u[k]; out.v[gi] = v[k]; out.w[gi] = w[k]; out.r[gi] = r[k];
            if (out.h != in.h) out.h[gi] = h[k];
            if (carry_out) {
                sc.carry_out[gi] = su[k];
                sc.carry_out[ncar + gi] = sv[k];
                sc.carry_out[2 * ncar + gi] = sfx[k];
                sc.carry_out[3 * ncar + gi] = sfy[k];
                sc.carry_out[4 * ncar + gi] = stz[k];
                sc.carry_out[5 * ncar + gi] = __uint_as_float(x0[k]);
                sc.carry_out[6 * ncar + gi] = __uint_as_float(y0[k]);
            }
        }
        // an empty cell of the group: zero moments
        if (t < ncg && S.cn[t] == 0 && !S.cskip[t]) {
            double *mo = sc.mom + (size_t)S.cc[t] * NMOM;
            for (int q = 0; q < NMOM; q++) mo[q] = 0.0;
        }
        if (__syncthreads_or(bad) && t == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
        bad = false;
        if (deep) atomicAdd(&sc.ctrl->deep, (unsigned long long)deep);
        deep = 0;
    }
}

// Fold the floes' running window sums into the window: a block per cell,
// the masses of the current state, fixed-order sums; the sums are cleared
// (the expansion centres are kept: they stay valid wherever the floes are).
__global__ void __launch_bounds__(128) k_carry_flush(DevState32 s, StepCommon sc, float *carry, long long ncarry)
{
    __shared__ double red[6][128];
    const int c = blockIdx.x, t = threadIdx.x;
    const int o = sc.off[c], n = sc.off[c + 1] - o;
    double a[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = t; i < n; i += 128) {
        const long long gi = o + i;
        const float r = s.r[gi], h = s.h[gi];
        const double m = (double)r * (double)r * (double)h;   // rho_ice pi cancels in the mean
        a[0] += m;
        a[1] += m * carry[gi];
        a[2] += m * carry[ncarry + gi];
        a[3] += carry[2 * ncarry + gi];
        a[4] += carry[3 * ncarry + gi];
        a[5] += carry[4 * ncarry + gi];
        for (int q = 0; q < 5; q++) carry[q * ncarry + gi] = 0.0f;
    }
    for (int q = 0; q < 6; q++) red[q][t] = a[q];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < 6; q++) red[q][t] += red[q][t + w];
        __syncthreads();
    }
    if (t == 0) {
        const int nc = sc.ncell;
        if (red[0][0] > 0.0) {
            sc.win[c] += red[1][0] / red[0][0];
            sc.win[nc + c] += red[2][0] / red[0][0];
        }
        sc.win[2 * nc + c] += red[3][0];
        sc.win[3 * nc + c] += red[4][0];
        sc.win[4 * nc + c] += red[5][0];
    }
}

}  // namespace

cudaError_t launch_carry_flush(const DevState32 &s, const StepCommon &sc, float *carry, long long ncarry,
                               cudaStream_t st)
{
    if (sc.ncell <= 0 || !carry) return cudaSuccess;
    k_carry_flush<<<sc.ncell, 128, 0, st>>>(s, sc, carry, ncarry);
    return cudaGetLastError();
}

size_t run_block_smem(int K) { return run_smem_bytes(K); }

cudaError_t run_block_prepare()
{
    const void *kern[3] = {(const void *)k_cell_run32_block<1>, (const void *)k_cell_run32_block<2>,
                           (const void *)k_cell_run32_block<4>};
    const size_t sm[3] = {run_smem_bytes(1), run_smem_bytes(2), run_smem_bytes(4)};
    for (int i = 0; i < 3; i++) {
        cudaError_t e = cudaFuncSetAttribute(kern[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Persistent grid of one class: as many blocks as fit on the device at once
// (at most one per group).
static int run_block_grid(int K, int ngroups)
{
    static int blocks_per_sm[3] = {0, 0, 0}, nsm = 0;
    const int ki = K == 1 ? 0 : (K == 2 ? 1 : 2);
    if (!blocks_per_sm[ki]) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        int b = 0;
        if (K == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cell_run32_block<1>, RT, run_smem_bytes(1));
        else if (K == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cell_run32_block<2>, RT, run_smem_bytes(2));
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cell_run32_block<4>, RT, run_smem_bytes(4));
        blocks_per_sm[ki] = b > 0 ? b : 1;
    }
    const int g = blocks_per_sm[ki] * (nsm > 0 ? nsm : 1);
    return g < ngroups ? g : ngroups;
}

cudaError_t launch_run_block(int K, const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                             const StepCommon &sc, const int4 *groups, int ngroups, const int4 *items, int qslot,
                             int nsteps, float skin_steps, cudaStream_t st)
{
    if (ngroups <= 0 || nsteps <= 0) return cudaSuccess;
    const int grid = run_block_grid(K, ngroups);
    if (K == 1)
        k_cell_run32_block<1><<<grid, RT, run_smem_bytes(1), st>>>(in, out, P, sc, groups, ngroups, items, qslot,
                                                                    nsteps, skin_steps);
    else if (K == 2)
        k_cell_run32_block<2><<<grid, RT, run_smem_bytes(2), st>>>(in, out, P, sc, groups, ngroups, items, qslot,
                                                                    nsteps, skin_steps);
    else
        k_cell_run32_block<4><<<grid, RT, run_smem_bytes(4), st>>>(in, out, P, sc, groups, ngroups, items, qslot,
                                                                    nsteps, skin_steps);
    return cudaGetLastError();
}

}  // namespace msd
