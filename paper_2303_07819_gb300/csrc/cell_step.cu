// cell_step.cu -- one fine step of every cell's doubly periodic DEM, fused
// with the per-cell moment reduction and the gradual coarse-to-fine update.
//
// Per cell (superparameterisation, Sec. 3.1): stage the cell's floes in shared
// memory, find all contacts within the cell under the cell-periodic minimum
// image, add the contact forces of Eq. (2.2) and the drag of Eq. (2.1c-d),
// advance by forward Euler, apply the gradual update of Sec. 3.3 on update
// steps, and reduce the post-step state to the cell's moments (Sec. 2.3) in
// FP64, accumulating the coarse-step window of Algorithm 1.
//
// One block owns one cell at a time, so the update is in place: the block
// reads its whole cell into shared memory before any thread writes.
#include <cmath>

#include "common.cuh"

namespace msd {

namespace {


// A large floe's search reach, capped at the cell side of its axis; NaN (a
// diverged state) takes the whole side.  Positions lie in [0, L), so the bin
// bounds derived from a capped reach stay within [-nb - 1, 2 nb + 1]: the
// integer width of the range cannot overflow, and a range narrower than the
// cell wraps into the bin table at most once on either side.
__device__ __forceinline__ float reach_cap(float reach, float L) { return reach < L ? reach : L; }

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Step facts shared by all blocks of a launch.
struct StepInfo {
    long long s;      // 1-based index of this step
    double t;         // time at the start of the step
    bool ramp;        // gradual-update step
    int ev;           // update index within the coarse step (1..N0/n_t)
};

__device__ __forceinline__ StepInfo step_info(const StepCommon &sc)
{
    StepInfo si;
    const Ctrl *ctrl = sc.ctrl;
    si.s = ctrl->base + sc.i_local + 1;
    si.t = (double)(si.s - 1) * sc.dt;
    const long long k = sc.i_local + 1;           // step within the coarse interval
    si.ramp = sc.couple && ctrl->have_tgt && (k % sc.n_t == 0);
    si.ev = (int)(k / sc.n_t);
    return si;
}


// Per-block copy of the step facts and the current cell's update, set by
// thread 0 (its FP64 arithmetic runs once per block, not once per thread).
struct BlockStep {
    float ua, va;          // wind at the start of the step
    int ramp, ev;
    float g, du, dv, dw;   // current cell's gradual update
};

__device__ __forceinline__ void block_step_init(BlockStep &bs, const StepCommon &sc, const Phys<float> &P)
{
    if (threadIdx.x == 0) {
        const StepInfo si = step_info(sc);
        float ua, va;
        wind_at(P, si.t, ua, va);
        bs.ua = ua;
        bs.va = va;
        bs.ramp = si.ramp;
        bs.ev = si.ev;
        bs.g = 1.0f;
        bs.du = bs.dv = bs.dw = 0.0f;
    }
    __syncthreads();
}

__device__ __forceinline__ void block_cell_ramp(BlockStep &bs, const StepCommon &sc, int c)
{
    if (threadIdx.x == 0 && bs.ramp) {
        const RampCell rc = ramp_cell(sc, c, bs.ev);
        bs.g = (float)rc.g;
        bs.du = (float)rc.du;
        bs.dv = (float)rc.dv;
        bs.dw = (float)rc.dw;
    }
}

// Work item of this block: a fixed item per block, or a ticket from the
// model's queue (persistent form).  The last block to leave resets the queue.
__device__ __forceinline__ int next_item(const StepCommon &sc, int persistent, int *sh_item, bool first)
{
    if (!persistent) return first ? (int)blockIdx.x : sc.ncell;
    __syncthreads();
    if (threadIdx.x == 0) {
        int it = (int)atomicAdd(&sc.ctrl->queue[0], 1u);
        if (it >= sc.ncell) {
            __threadfence();
            unsigned done = atomicAdd(&sc.ctrl->queue[1], 1u);
            if (done == gridDim.x - 1) {
                sc.ctrl->queue[0] = 0u;
                sc.ctrl->queue[1] = 0u;
                __threadfence();
            }
        }
        *sh_item = it;
    }
    __syncthreads();
    return *sh_item;
}

// Block reduction of the per-thread moment partials; thread 0 writes the cell
// moments and adds the window sums (Algorithm 1: mass-weighted mean velocity
// and total drag of each fine step).
template <class R, int T>
__device__ __forceinline__ void reduce_write(R (&acc)[NMOM], double *red, const StepCommon &sc,
                                             int c, int n)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 1; k < NMOM; k++) {
        R v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * NMOM + k] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m[NMOM];
        m[0] = (double)n;
        for (int k = 1; k < NMOM; k++) {
            double s = 0.0;
            for (int w = 0; w < T / 32; w++) s += red[w * NMOM + k];
            m[k] = s;
        }
        double *mo = sc.mom + (size_t)c * NMOM;
        for (int k = 0; k < NMOM; k++) mo[k] = m[k];
        if (sc.couple) {
            const int nc = sc.ncell;
            if (m[1] > 0.0) {
                sc.win[c] += m[2] / m[1];
                sc.win[nc + c] += m[3] / m[1];
            }
            sc.win[2 * nc + c] += m[9];
            sc.win[3 * nc + c] += m[10];
            sc.win[4 * nc + c] += m[11];
        }
    }
}

template <class R>
__device__ __forceinline__ void add_moments(R (&acc)[NMOM], const R mass_c, const R inertia_f,
                                            R u, R v, R w, R r, R h, R Fx, R Fy, R T)
{
    const R m = mass_c * r * r * h;
    const R I = inertia_f * m * r * r;
    acc[1] += m;
    acc[2] += m * u;
    acc[3] += m * v;
    acc[4] += I;
    acc[5] += I * w;
    acc[6] += R(3.14159265358979323846) * r * r;
    acc[7] += m * u * u;
    acc[8] += m * v * v;
    acc[9] += Fx;
    acc[10] += Fy;
    acc[11] += T;
}

// ===================================================================== FP32
// Positions are 32-bit fixed point of the periodic cell (2^32 = cell side), so
// the periodic wrap after the step and the minimum image of a pair are plain
// 32-bit integer wrap-around.

template <int T>
__global__ void __launch_bounds__(T)
k_cell_step32_brute(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, int persistent)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int maxn = sc.max_n;
    float4 *A = reinterpret_cast<float4 *>(smem);                  // r, h, u, v
    uint2 *Qp = reinterpret_cast<uint2 *>(smem + align16(sizeof(float4) * maxn));
    float *W = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(Qp) + align16(sizeof(uint2) * maxn));
    double *red = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(W) + align16(sizeof(float) * maxn));
    float *base = reinterpret_cast<float *>(red + (T / 32) * NMOM);
    int *sh_item = reinterpret_cast<int *>(base + MAXM);

    __shared__ BlockStep bs;
    block_step_init(bs, sc, P);
    const float dt = sc.k.dt;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    unsigned deep = 0;
    bool bad = false;

    for (int item = next_item(sc, persistent, sh_item, true); item < sc.ncell;
         item = next_item(sc, persistent, sh_item, false)) {
        const int c = sc.order[item];
        const int o = sc.off[c], n = sc.off[c + 1] - o;
        const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;
        if (threadIdx.x < P.n_modes) {
            const int m = threadIdx.x;
            base[threadIdx.x] = corner_phase(P, m, ix, iy, sc.g.nx, sc.g.nyr, inx, iny);
        }
        for (int k = threadIdx.x; k < n; k += T) {
            A[k] = make_float4(in.r[o + k], in.h[o + k], in.u[o + k], in.v[o + k]);
            Qp[k] = make_uint2(in.xq[o + k], in.yq[o + k]);
            W[k] = in.w[o + k];
        }
        block_cell_ramp(bs, sc, c);
        __syncthreads();

        float acc[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; k++) acc[k] = 0.0f;

        for (int l = threadIdx.x; l < n; l += T) {
            const float4 al = A[l];
            const uint2 ql = Qp[l];
            const float wl = W[l];
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            for (int j = 0; j < n; j++) {
                if (j == l) continue;
                const uint2 qj = Qp[j];
                const float dx = (float)(int)(qj.x - ql.x) * sx;
                const float dy = (float)(int)(qj.y - ql.y) * sy;
                const float d2 = dx * dx + dy * dy;
                const float4 aj = A[j];
                const float S = al.x + aj.x;
                if (d2 < S * S) {
                    contact_add(dx, dy, d2, al.x, aj.x, al.y, aj.y, aj.z - al.z, aj.w - al.w, wl,
                                W[j], P, fx, fy, tq, deep);
                }
            }
            // forcing at the floe's global position (reading: cell origin + local)
            const float xf = (float)ql.x * INV2_32F, yf = (float)ql.y * INV2_32F;
            float uo, vo, zeta;
            ocean_f32(P, base, inx, iny, xf, yf, uo, vo, zeta);
            float Fdx, Fdy, Td;
            drag_force(P, uo, vo, zeta, bs.ua, bs.va, al.z, al.w, wl, al.x, Fdx, Fdy, Td);
            fx += Fdx; fy += Fdy; tq += Td;
            // forward Euler with every right-hand side at t_n
            const float r = al.x, h = al.y;
            const float m = P.mass_c * r * r * h;
            const float I = P.inertia_f * m * r * r;
            const uint32_t xn = ql.x + (uint32_t)__float2int_rn(dt * al.z * isx);
            const uint32_t yn = ql.y + (uint32_t)__float2int_rn(dt * al.w * isy);
            float th = in.th[o + l] + dt * wl;
            float un = al.z + dt * (fx / m);
            float vn = al.w + dt * (fy / m);
            float wn = wl + dt * (tq / I);
            float rn = r;
            if (bs.ramp) {
                rn = r * bs.g;
                un += bs.du;
                vn += bs.dv;
                wn += bs.dw;
            }
            bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
            out.xq[o + l] = xn;
            out.yq[o + l] = yn;
            out.th[o + l] = th;
            out.u[o + l] = un;
            out.v[o + l] = vn;
            out.w[o + l] = wn;
            if (bs.ramp || out.r != in.r) out.r[o + l] = rn;
            add_moments(acc, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
        }
        reduce_write<float, T>(acc, red, sc, c, n);
        __syncthreads();
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&sc.ctrl->deep, 1ull);
}

// ============================================================= FP32 binned
// Pair search with a per-cell bin grid in shared memory.  With nb bins per
// side (nb ~ sqrt(n) / beta, 3 <= nb <= nbmax) of side B, a floe is "small"
// when r <= B/2: two small floes in contact have centres less than B apart,
// so a small floe finds its small partners in the 3 x 3 bins around its own.
// Each neighbouring bin is visited with the periodic shift of the cell that
// brings it next to the floe, so the pair test needs no minimum image.  The
// few large floes form one list that every floe scans with a float minimum
// image; a large floe finds its small partners in the bins within its reach.
// Every floe sums its own contacts (each pair is evaluated from both sides),
// so no atomics touch forces and results do not depend on thread timing.
// The bin test runs on float cell-local positions; the force of a contact
// uses the exact 32-bit fixed-point separation.  Bin contents are sorted by
// floe index, so the summation order is fixed.

template <int T>
__device__ __forceinline__ int block_scan_excl(const int *in, int *out, int count, int *tmp)
{
    const int per = (count + T - 1) / T;
    const int b = threadIdx.x * per;
    const int e = min(b + per, count);
    int s = 0;
    for (int i = b; i < e; i++) s += in[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < T / 32; w++) {
            const int t = tmp[w];
            tmp[w] = acc;
            acc += t;
        }
        tmp[T / 32] = acc;
    }
    __syncthreads();
    int run = tmp[warp] + x - s;
    for (int i = b; i < e; i++) {
        const int v = in[i];
        out[i] = run;
        run += v;
    }
    const int total = tmp[T / 32];
    __syncthreads();
    return total;
}

// float minimum image for a separation in (-L, L): subtract L * rint(d / L),
// rint by the 1.5 * 2^23 rounding constant (round to nearest, FMA pipe only)
__device__ __forceinline__ float min_image(float d, float L, float iL)
{
    const float k = __fsub_rn(__fadd_rn(d * iL, 12582912.0f), 12582912.0f);
    return fmaf(-k, L, d);
}

constexpr int MAXC_B = 16;   // contacts a thread collects before computing their forces

struct Bin32 {
    float4 *P4;     // x, y (m, cell-local float), r, h          [index order]
    float4 *V4;     // u, v, w                                   [index order]
    float4 *S4;     // P4 in search order: small floes by bin, then large floes
    float4 *F4;     // force x, y, torque                        [index order]
    uint2 *Q;       // exact fixed-point position                [index order]
    int *cnt;       // [nb^2 + 1] bin counts, then cursors
    int *bst;       // [nb^2 + 1] bin starts
    short *sidx;    // search position -> floe index
    short *bin;     // floe index -> bin (-1: large)
    short *clist;   // [MAXC_B][T] contact candidates per thread
    int *tmp;       // scan scratch
    double *red;
    float *base;
    int *misc;
};

template <int T>
__device__ __forceinline__ Bin32 carve32(unsigned char *smem, int maxn, int nbmax)
{
    Bin32 b;
    const int nbins = nbmax * nbmax + 1;
    size_t o = 0;
    b.P4 = reinterpret_cast<float4 *>(smem + o); o += align16(sizeof(float4) * maxn);
    b.V4 = reinterpret_cast<float4 *>(smem + o); o += align16(sizeof(float4) * maxn);
    b.S4 = reinterpret_cast<float4 *>(smem + o); o += align16(sizeof(float4) * maxn);
    b.F4 = reinterpret_cast<float4 *>(smem + o); o += align16(sizeof(float4) * maxn);
    b.Q = reinterpret_cast<uint2 *>(smem + o); o += align16(sizeof(uint2) * maxn);
    b.red = reinterpret_cast<double *>(smem + o); o += align16(sizeof(double) * (T / 32) * NMOM);
    b.cnt = reinterpret_cast<int *>(smem + o); o += align16(sizeof(int) * nbins);
    b.bst = reinterpret_cast<int *>(smem + o); o += align16(sizeof(int) * nbins);
    b.tmp = reinterpret_cast<int *>(smem + o); o += align16(sizeof(int) * (T / 32 + 1));
    b.base = reinterpret_cast<float *>(smem + o); o += align16(sizeof(float) * MAXM);
    b.misc = reinterpret_cast<int *>(smem + o); o += align16(sizeof(int) * 8);
    b.sidx = reinterpret_cast<short *>(smem + o); o += align16(sizeof(short) * maxn);
    b.bin = reinterpret_cast<short *>(smem + o); o += align16(sizeof(short) * maxn);
    b.clist = reinterpret_cast<short *>(smem + o); o += align16(sizeof(short) * MAXC_B * T);
    return b;
}

__host__ __device__ inline size_t smem32_binned(int T, int maxn, int nbmax)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const int nbins = nbmax * nbmax + 1;
    return 4 * a16(sizeof(float4) * maxn) + a16(sizeof(uint2) * maxn) + a16(sizeof(double) * (T / 32) * NMOM) +
           2 * a16(sizeof(int) * nbins) + a16(sizeof(int) * (T / 32 + 1)) + a16(sizeof(float) * MAXM) +
           a16(sizeof(int) * 8) + 2 * a16(sizeof(short) * maxn) + a16(sizeof(short) * MAXC_B * T);
}

// ---- candidate lists (variant 4): recording and walking a floe's list

// half h (0..7) of a 16-byte list group
__device__ __forceinline__ int list_half(const uint4 &g, int h)
{
    const uint32_t w = h < 2 ? g.x : (h < 4 ? g.y : (h < 6 ? g.z : g.w));
    return (int)((h & 1) ? (w >> 16) : (w & 0xffffu));
}

// A floe's list as the search finds its candidates: the head in registers,
// entries past it straight to the floe's tail groups.
struct ListRec {
    uint32_t h0 = 0u, h1 = 0u, h2 = 0u, h3 = 0u;
    int nlst = 0;
    __device__ __forceinline__ void add(uint16_t *tail16, int j)
    {
        if (nlst < NLH) {
            const int s = nlst + 1;   // half 0 holds the count
            const uint32_t v = (uint32_t)j << ((s & 1) * 16);
            const int wd = s >> 1;
            h0 |= wd == 0 ? v : 0u;
            h1 |= wd == 1 ? v : 0u;
            h2 |= wd == 2 ? v : 0u;
            h3 |= wd == 3 ? v : 0u;
        } else if (nlst < NBL) {
            tail16[nlst - NLH] = (uint16_t)j;
        }
        nlst++;
    }
    __device__ __forceinline__ uint4 head() const
    {
        return make_uint4(h0 | (uint32_t)(nlst < NBL ? nlst : NBL), h1, h2, h3);
    }
};

// Calls pair(load(j)) for the entries j of a floe's list in order, from one
// call site (every candidate gets the same compiled arithmetic).  The next
// entry's partner is loaded before the current pair is computed, and the
// next tail group one group ahead of its use.
template <class LoadF, class PairF>
__device__ __forceinline__ void list_walk(const uint4 hd, const uint4 *tl, LoadF &&load, PairF &&pair)
{
    const int cnt = (int)(hd.x & 0xffffu);
    if (cnt == 0) return;
    uint4 g = hd, nx = make_uint4(0u, 0u, 0u, 0u);
    if (cnt > NLH) nx = tl[0];
    int h = 2, gi = 1;   // half of the next entry to load (entry 0 is half 1 of the head)
    auto cur = load(list_half(g, 1));
    for (int t = 0; t < cnt; t++) {
        auto nxt = cur;
        if (t + 1 < cnt) {
            if (h == 8) {
                g = nx;
                h = 0;
                if (NLH + 8 * gi < cnt) nx = tl[gi];
                gi++;
            }
            nxt = load(list_half(g, h));
            h++;
        }
        pair(cur);
        cur = nxt;
    }
}

// a list entry's partner as staged in shared memory
struct Partner {
    uint2 q;     // fixed-point position
    float4 p;    // x, y, r, h
    float4 v;    // u, v, w, (theta)
};

// LISTS: variant 4's candidate lists (see k_cell_step32_wlist) kept across
// steps; a cell rebuilds them with this kernel's binned search, widened by
// the skin, and otherwise tests only its lists.
template <int T, bool LISTS = false>
__global__ void __launch_bounds__(T)
k_cell_step32_binned(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, float beta, int item0,
                     int item1, int maxn, int nbmax, int seg)
{
    __shared__ float s_vmax[T / 32];
    extern __shared__ __align__(16) unsigned char smem[];
    const Bin32 sm = carve32<T>(smem, maxn, nbmax);

    __shared__ BlockStep bs;
    block_step_init(bs, sc, P);
    const float dt = sc.k.dt;
    const float Lx = sc.k.Lx, Ly = sc.k.Ly, iLx = sc.k.iLx, iLy = sc.k.iLy;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    unsigned deep = 0;
    bool bad = false;

    if (sc.live) item1 = min(item1, item0 + sc.live[seg]);
    for (int item = item0 + blockIdx.x; item < item1; item += gridDim.x) {
        const int c = sc.order[item];
        const int o = sc.off[c], n = sc.off[c + 1] - o;
        const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;
        // ---- candidate lists: keep them or rebuild (block-uniform decision)
        bool rebuild = true;
        float skin = 0.0f;
        uint4 hn = make_uint4(0u, 0u, 0u, 0u);     // list head of this thread's next floe
        const long long sstep = sc.ctrl->base + sc.i_local + 1;
        int nb = (int)(sqrtf((float)n) / beta);
        nb = nb > nbmax ? nbmax : nb;
        if (nb < 3) nb = 0;                       // few floes: every floe in the list
        const float Bx = nb ? Lx / nb : Lx, By = nb ? Ly / nb : Ly;
        const int nbins = nb * nb;
        if (threadIdx.x < P.n_modes) {
            const int m = threadIdx.x;
            sm.base[m] = corner_phase(P, m, ix, iy, sc.g.nx, sc.g.nyr, inx, iny);
        }
        for (int b = threadIdx.x; b <= nbins; b += T) sm.cnt[b] = 0;
        if (LISTS) {
            // ---- stage the cell, and decide whether the lists still hold:
            // one pass, all of a floe's loads independent
            const long long built = sc.nl.cstep[c];
            const float lim = 0.25f * sc.nl.skin[c] * sc.nl.skin[c];
            const bool r0 = (sc.i_local % sc.n_t == 0) || built < 0 || sstep - built >= sc.n_t || sstep < built;
            if (!r0 && (int)threadIdx.x < n) hn = sc.nl.head[o + threadIdx.x];
            block_cell_ramp(bs, sc, c);      // read after the barrier below
            bool far = false;
            float vmax = 0.0f;
            for (int k = threadIdx.x; k < n; k += T) {
                const uint2 b = sc.nl.xb[o + k];
                const uint32_t xq = in.xq[o + k], yq = in.yq[o + k];
                const float r = in.r[o + k], h = in.h[o + k], u = in.u[o + k], v = in.v[o + k], w = in.w[o + k];
                sm.P4[k] = make_float4((float)xq * sx, (float)yq * sy, r, h);
                sm.V4[k] = make_float4(u, v, w, 0.0f);
                sm.Q[k] = make_uint2(xq, yq);
                const float dx = (float)(int)(xq - b.x) * sx, dy = (float)(int)(yq - b.y) * sy;
                far |= dx * dx + dy * dy > lim;
                vmax = fmaxf(vmax, fmaxf(fabsf(u), fabsf(v)));
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, d));
            if ((threadIdx.x & 31) == 0) s_vmax[threadIdx.x >> 5] = vmax;
            rebuild = __syncthreads_or(r0 || far) != 0;
            for (int w = 0; w < T / 32; w++) vmax = fmaxf(vmax, s_vmax[w]);
            // as in k_cell_step32_wlist
            if (rebuild) skin = 4.0f * vmax * dt * (float)sc.n_t + 1.0e-3f;
        } else {
            __syncthreads();
        }
        const float Rs = nb ? 0.5f * fminf(Bx, By) - 0.5f * skin : -1.0f;
        if (LISTS) {
            // ---- bins from the staged cell (only when searching again)
            if (rebuild) {
                for (int k = threadIdx.x; k < n; k += T) {
                    const uint2 q = sm.Q[k];
                    short b = -1;
                    if (sm.P4[k].z <= Rs) {
                        b = (short)(__umulhi(q.y, (unsigned)nb) * nb + __umulhi(q.x, (unsigned)nb));
                        atomicAdd(&sm.cnt[b], 1);
                    }
                    sm.bin[k] = b;
                    sc.nl.xb[o + k] = q;
                }
            }
        } else {
            // ---- stage the cell and count small floes per bin
            for (int k = threadIdx.x; k < n; k += T) {
                const uint32_t xq = in.xq[o + k], yq = in.yq[o + k];
                const float r = in.r[o + k];
                sm.P4[k] = make_float4((float)xq * sx, (float)yq * sy, r, in.h[o + k]);
                sm.V4[k] = make_float4(in.u[o + k], in.v[o + k], in.w[o + k], 0.0f);
                sm.Q[k] = make_uint2(xq, yq);
                short b = -1;
                if (r <= Rs) {
                    b = (short)(__umulhi(yq, (unsigned)nb) * nb + __umulhi(xq, (unsigned)nb));
                    atomicAdd(&sm.cnt[b], 1);
                }
                sm.bin[k] = b;
            }
        }
        if (!(LISTS && !rebuild)) {
        __syncthreads();
        const int nsmall = block_scan_excl<T>(sm.cnt, sm.bst, nbins + 1, sm.tmp);
        for (int b = threadIdx.x; b <= nbins; b += T) sm.cnt[b] = 0;
        __syncthreads();
        // ---- small floes to their bins; large floes, in index order, after them
        int run = nsmall;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int k0 = 0; k0 < n; k0 += T) {
            const int k = k0 + threadIdx.x;
            const bool valid = k < n;
            const short b = valid ? sm.bin[k] : (short)0;
            if (valid && b >= 0) sm.sidx[sm.bst[b] + atomicAdd(&sm.cnt[b], 1)] = (short)k;
            const bool large = valid && b < 0;
            const unsigned bal = __ballot_sync(0xffffffffu, large);
            if (lane == 0) sm.tmp[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < T / 32; w++) {
                const int t = sm.tmp[w];
                before += (w < warp) ? t : 0;
                total += t;
            }
            if (large) sm.sidx[run + before + __popc(bal & ((1u << lane) - 1u))] = (short)k;
            run += total;
            __syncthreads();
        }
        // ---- fixed order inside each bin: ascending floe index
        for (int b = threadIdx.x; b < nbins; b += T) {
            const int s0 = sm.bst[b], e0 = sm.bst[b + 1];
            for (int i = s0 + 1; i < e0; i++) {
                const short key = sm.sidx[i];
                int j = i - 1;
                while (j >= s0 && sm.sidx[j] > key) {
                    sm.sidx[j + 1] = sm.sidx[j];
                    j--;
                }
                sm.sidx[j + 1] = key;
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += T) sm.S4[p] = sm.P4[sm.sidx[p]];
        __syncthreads();

        // ---- contacts (and, with lists, every candidate within the skin recorded)
        bool overflow = false;
        for (int p = threadIdx.x; p < n; p += T) {
            const int l = sm.sidx[p];
            const float4 pl = sm.P4[l];
            const float4 vl = sm.V4[l];
            const uint2 ql = sm.Q[l];
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            ListRec rec;
            uint16_t *tail16 = LISTS ? reinterpret_cast<uint16_t *>(sc.nl.tail + (size_t)(o + l) * NLT) : nullptr;
            auto touch = [&](int k) {
                const int j = sm.sidx[k];
                const uint2 qj = sm.Q[j];
                const float dx = (float)(int)(qj.x - ql.x) * sx;
                const float dy = (float)(int)(qj.y - ql.y) * sy;
                const float4 pj = sm.P4[j];
                const float4 vj = sm.V4[j];
                contact_add(dx, dy, dx * dx + dy * dy, pl.z, pj.z, pl.w, pj.w, vj.x - vl.x, vj.y - vl.y, vl.z,
                            vj.z, P, fx, fy, tq, deep);
                if (LISTS) rec.add(tail16, j);
            };
            // collect candidates, then compute their forces with the threads in step
            int ncand = 0;
            short *cl = sm.clist + threadIdx.x;
            auto flush = [&]() {
                for (int i = 0; i < ncand; i++) touch(cl[T * i]);
                ncand = 0;
            };
            auto hit = [&](int k) {
                if (ncand == MAXC_B) flush();
                cl[T * ncand] = (short)k;
                ncand++;
            };
            // small partners through the bins
            int bx0, bx1, by0, by1;
            if (p < nsmall) {
                const int b = sm.bin[l];
                const int bx = b % nb, by = b / nb;
                bx0 = bx - 1; bx1 = bx + 1; by0 = by - 1; by1 = by + 1;
            } else if (nb) {
                const float reach = 1.001f * (pl.z + Rs + skin);
                const float rx = reach_cap(reach, Lx), ry = reach_cap(reach, Ly);
                bx0 = (int)floorf((pl.x - rx) / Bx); bx1 = (int)floorf((pl.x + rx) / Bx);
                by0 = (int)floorf((pl.y - ry) / By); by1 = (int)floorf((pl.y + ry) / By);
                if (bx1 - bx0 + 1 >= nb) { bx0 = 0; bx1 = nb - 1; }
                if (by1 - by0 + 1 >= nb) { by0 = 0; by1 = nb - 1; }
            } else {
                bx0 = 0; bx1 = -1; by0 = 0; by1 = -1;
            }
            const bool wrapx = (bx0 == 0 && bx1 == nb - 1 && p >= nsmall);
            const bool wrapy = (by0 == 0 && by1 == nb - 1 && p >= nsmall);
            for (int by = by0; by <= by1; by++) {
                const int wy = by < 0 ? by + nb : (by >= nb ? by - nb : by);
                const float ys = wrapy ? pl.y : (by < 0 ? pl.y + Ly : (by >= nb ? pl.y - Ly : pl.y));
                for (int bx = bx0; bx <= bx1; bx++) {
                    const int wx = bx < 0 ? bx + nb : (bx >= nb ? bx - nb : bx);
                    const float xs = wrapx ? pl.x : (bx < 0 ? pl.x + Lx : (bx >= nb ? pl.x - Lx : pl.x));
                    const int wb = wy * nb + wx;
                    const int e0 = sm.bst[wb + 1];
                    for (int k = sm.bst[wb]; k < e0; k++) {
                        const float4 q = sm.S4[k];
                        float dx = q.x - xs, dy = q.y - ys;
                        if (wrapx) dx = min_image(dx, Lx, iLx);
                        if (wrapy) dy = min_image(dy, Ly, iLy);
                        const float S = pl.z + q.z + skin;
                        if (k != p && dx * dx + dy * dy < S * S) hit(k);
                    }
                }
            }
            // large partners through the list
            for (int k = nsmall; k < n; k++) {
                const float4 q = sm.S4[k];
                const float dx = min_image(q.x - pl.x, Lx, iLx);
                const float dy = min_image(q.y - pl.y, Ly, iLy);
                const float S = pl.z + q.z + skin;
                if (k != p && dx * dx + dy * dy < S * S) hit(k);
            }
            flush();
            sm.F4[l] = make_float4(fx, fy, tq, 0.0f);
            if (LISTS) {
                sc.nl.head[o + l] = rec.head();
                overflow |= rec.nlst > NBL;
            }
        }
        if (LISTS) {
            const bool any_over = __syncthreads_or(overflow) != 0;
            if (threadIdx.x == 0) {
                sc.nl.cstep[c] = any_over ? -1 : sstep;   // an overflowing cell searches again next step
                sc.nl.skin[c] = skin;
            }
        }
        }
        if (!LISTS) block_cell_ramp(bs, sc, c);
        if (!(LISTS && !rebuild)) __syncthreads();   // the search's forces come from other threads

        // ---- contact forces from the lists (each thread its own floes: no
        // barrier; the next floe's head is loaded while this floe's candidates
        // are tested) or from the search above; then drag, forward Euler,
        // gradual update, moments (index order: coalesced I/O)
        float acc[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; k++) acc[k] = 0.0f;
        for (int l = threadIdx.x; l < n; l += T) {
            const float4 pl = sm.P4[l];
            const float4 vl = sm.V4[l];
            const uint2 ql = sm.Q[l];
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            if (LISTS && !rebuild) {
                const uint4 hd = hn;
                if (l + T < n) hn = sc.nl.head[o + l + T];
                list_walk(
                    hd, sc.nl.tail + (size_t)(o + l) * NLT,
                    [&](int j) { return Partner{sm.Q[j], sm.P4[j], sm.V4[j]}; },
                    [&](const Partner &b) {
                        const float dx = (float)(int)(b.q.x - ql.x) * sx;
                        const float dy = (float)(int)(b.q.y - ql.y) * sy;
                        contact_add(dx, dy, dx * dx + dy * dy, pl.z, b.p.z, pl.w, b.p.w, b.v.x - vl.x, b.v.y - vl.y,
                                    vl.z, b.v.z, P, fx, fy, tq, deep);
                    });
            } else {
                const float4 f4 = sm.F4[l];
                fx = f4.x; fy = f4.y; tq = f4.z;
            }
            const float xf = (float)ql.x * INV2_32F, yf = (float)ql.y * INV2_32F;
            float uo, vo, zeta;
            ocean_f32(P, sm.base, inx, iny, xf, yf, uo, vo, zeta);
            float Fdx, Fdy, Td;
            drag_force(P, uo, vo, zeta, bs.ua, bs.va, vl.x, vl.y, vl.z, pl.z, Fdx, Fdy, Td);
            fx += Fdx; fy += Fdy; tq += Td;
            const float r = pl.z, h = pl.w;
            const float m = P.mass_c * r * r * h;
            const float I = P.inertia_f * m * r * r;
            const uint32_t xn = ql.x + (uint32_t)__float2int_rn(dt * vl.x * isx);
            const uint32_t yn = ql.y + (uint32_t)__float2int_rn(dt * vl.y * isy);
            const float th = in.th[o + l] + dt * vl.z;
            float un = vl.x + dt * (fx / m);
            float vn = vl.y + dt * (fy / m);
            float wn = vl.z + dt * (tq / I);
            float rn = r;
            if (bs.ramp) {
                rn = r * bs.g;
                un += bs.du;
                vn += bs.dv;
                wn += bs.dw;
            }
            bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
            out.xq[o + l] = xn;
            out.yq[o + l] = yn;
            out.th[o + l] = th;
            out.u[o + l] = un;
            out.v[o + l] = vn;
            out.w[o + l] = wn;
            if (bs.ramp || out.r != in.r) out.r[o + l] = rn;
            add_moments(acc, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
        }
        reduce_write<float, T>(acc, sm.red, sc, c, n);
        __syncthreads();
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&sc.ctrl->deep, 1ull);
}

// =============================================================== FP32 warp
// One warp owns one cell (cells of up to 256 floes): no block barriers, a
// lane per floe.  The cell is stored in shared memory in search order (small
// floes by bin, ascending floe index within a bin; then large floes in index
// order).  The rank of a floe inside its bin comes from __match_any_sync, so
// placement needs neither atomics nor a sort and the order is deterministic.
// The same lane finds a floe's contacts and advances it, so the force stays
// in registers; the floe is written back to its own global slot.

constexpr int MAXC = 12;   // contacts a lane collects before computing their forces

__host__ __device__ inline size_t warp_region_bytes(int cap, int nbmax)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    return 2 * a16(sizeof(float4) * cap) + a16(sizeof(uint2) * cap) + a16(sizeof(short) * cap) +
           a16(sizeof(short) * MAXC * 32) + 2 * a16(sizeof(int) * (nbmax * nbmax + 1)) + a16(sizeof(float2) * MAXM);
}

struct WarpSm {
    float4 *S4;    // x, y (m, float), r, h
    float4 *SV;    // u, v, w, theta
    uint2 *SQ;     // exact fixed-point position
    short *orig;   // floe index within the cell
    int *cnt, *bst;
    short *clist;       // [MAXC][32] contact candidates per lane
    float2 *Cm;    // per mode: (cos, sin) of the cell's phase, or (phase, -) without the small-angle form
};

__device__ __forceinline__ WarpSm carve_warp(unsigned char *p, int cap, int nbmax)
{
    WarpSm w;
    size_t o = 0;
    w.S4 = reinterpret_cast<float4 *>(p + o); o += align16(sizeof(float4) * cap);
    w.SV = reinterpret_cast<float4 *>(p + o); o += align16(sizeof(float4) * cap);
    w.SQ = reinterpret_cast<uint2 *>(p + o); o += align16(sizeof(uint2) * cap);
    w.orig = reinterpret_cast<short *>(p + o); o += align16(sizeof(short) * cap);
    w.clist = reinterpret_cast<short *>(p + o); o += align16(sizeof(short) * MAXC * 32);
    w.cnt = reinterpret_cast<int *>(p + o); o += align16(sizeof(int) * (nbmax * nbmax + 1));
    w.bst = reinterpret_cast<int *>(p + o); o += align16(sizeof(int) * (nbmax * nbmax + 1));
    w.Cm = reinterpret_cast<float2 *>(p + o);
    return w;
}


// exclusive scan of in[0..count) into out by one warp; returns the total
__device__ __forceinline__ int warp_scan_excl(const int *in, int *out, int count, int lane)
{
    const int per = (count + 31) >> 5;
    const int b = lane * per, e = min(b + per, count);
    int s = 0;
    for (int i = b; i < e; i++) s += in[i];
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);
    int run = x - s;
    for (int i = b; i < e; i++) {
        const int v = in[i];
        out[i] = run;
        run += v;
    }
    __syncwarp();
    return total;
}

// Warp sum of 16 values by halving exchanges (16 shuffles in all): lanes 2k
// and 2k+1 end with the total of value k.
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane)
{
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int half = 8 >> r;          // values kept after this round
        const int off = 16 >> r;          // lane distance
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 8)
k_cell_step32_warp(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, float beta, int item0,
                   int item1, int cap, int nbmax, int seg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockStep bs;
    block_step_init(bs, sc, P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = item0 + blockIdx.x * WARPS + warp;
    if (sc.live) item1 = min(item1, item0 + sc.live[seg]);
    if (item >= item1) return;
    const WarpSm sm = carve_warp(smem + warp * warp_region_bytes(cap, nbmax), cap, nbmax);
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;

    const float dt = sc.k.dt;
    const float Lx = sc.k.Lx, Ly = sc.k.Ly, iLx = sc.k.iLx, iLy = sc.k.iLy;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    const int c = sc.order[item];
    const int o = sc.off[c], n = sc.off[c + 1] - o;
    const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;

    float rg = 1.0f, rdu = 0.0f, rdv = 0.0f, rdw = 0.0f;
    if (bs.ramp) {
        if (lane == 0) {
            const RampCell rc = ramp_cell(sc, c, bs.ev);
            rg = (float)rc.g; rdu = (float)rc.du; rdv = (float)rc.dv; rdw = (float)rc.dw;
        }
        rg = __shfl_sync(FULL, rg, 0); rdu = __shfl_sync(FULL, rdu, 0);
        rdv = __shfl_sync(FULL, rdv, 0); rdw = __shfl_sync(FULL, rdw, 0);
    }
    if (lane < P.n_modes) {
        const int m = lane;
        const float b = corner_phase(P, m, ix, iy, sc.g.nx, sc.g.nyr, inx, iny);
        float sn, cs;
        if (P.taylor) {
            sincospif(2.0f * b, &sn, &cs);
            sm.Cm[m] = make_float2(cs, sn);
        } else {
            sm.Cm[m] = make_float2(b, 0.0f);
        }
    }

    int nb = (int)(sqrtf((float)n) / beta);
    nb = nb > nbmax ? nbmax : nb;
    if (nb < 3) nb = 0;
    const float Bx = nb ? Lx / nb : Lx, By = nb ? Ly / nb : Ly;
    const float Rs = nb ? 0.5f * fminf(Bx, By) : -1.0f;
    const int nbins = nb * nb;
    for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
    __syncwarp();

    // ---- count small floes per bin
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < n;
        const uint32_t xq = valid ? in.xq[o + k] : 0u, yq = valid ? in.yq[o + k] : 0u;
        const float r = valid ? in.r[o + k] : 0.0f;
        const bool small = valid && r <= Rs;
        const int b = small ? (int)(__umulhi(yq, (unsigned)nb) * nb + __umulhi(xq, (unsigned)nb)) : -1 - lane;
        const unsigned m = __match_any_sync(FULL, b);
        if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
        __syncwarp();
    }
    const int nsmall = warp_scan_excl(sm.cnt, sm.bst, nbins + 1, lane);
    for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
    __syncwarp();
    // ---- place every floe at its search position
    int lrun = nsmall;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < n;
        uint32_t xq = 0u, yq = 0u;
        float r = 0.0f, h = 0.0f, u = 0.0f, v = 0.0f, w = 0.0f, th = 0.0f;
        if (valid) {
            xq = in.xq[o + k]; yq = in.yq[o + k];
            r = in.r[o + k]; h = in.h[o + k];
            u = in.u[o + k]; v = in.v[o + k]; w = in.w[o + k]; th = in.th[o + k];
        }
        const bool small = valid && r <= Rs;
        const bool large = valid && !small;
        const int b = small ? (int)(__umulhi(yq, (unsigned)nb) * nb + __umulhi(xq, (unsigned)nb)) : -1 - lane;
        const unsigned m = __match_any_sync(FULL, b);
        const unsigned bl = __ballot_sync(FULL, large);
        int pos = 0;
        if (small) pos = sm.bst[b] + sm.cnt[b] + __popc(m & lt);
        else if (large) pos = lrun + __popc(bl & lt);
        if (valid) {
            sm.S4[pos] = make_float4((float)xq * sx, (float)yq * sy, r, h);
            sm.SV[pos] = make_float4(u, v, w, 0.0f);
            sm.SQ[pos] = make_uint2(xq, yq);
            sm.orig[pos] = (short)k;
            // forward Euler for position and angle needs only this floe's old
            // state: write them now (the cell's old positions live in SQ)
            out.xq[o + k] = xq + (uint32_t)__float2int_rn(dt * u * isx);
            out.yq[o + k] = yq + (uint32_t)__float2int_rn(dt * v * isy);
            out.th[o + k] = th + dt * w;
        }
        __syncwarp();
        if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
        lrun += __popc(bl);
        __syncwarp();
    }

    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = 0.0f;
    unsigned deep = 0;
    bool bad = false;
    for (int p = lane; p < n; p += 32) {
        const float4 pl = sm.S4[p];
        const float4 vl = sm.SV[p];
        const uint2 ql = sm.SQ[p];
        float fx = 0.0f, fy = 0.0f, tq = 0.0f;
        auto touch = [&](int k) {
            const uint2 qj = sm.SQ[k];
            const float dx = (float)(int)(qj.x - ql.x) * sx;
            const float dy = (float)(int)(qj.y - ql.y) * sy;
            const float4 pj = sm.S4[k];
            const float4 vj = sm.SV[k];
            contact_add(dx, dy, dx * dx + dy * dy, pl.z, pj.z, pl.w, pj.w, vj.x - vl.x, vj.y - vl.y, vl.z, vj.z,
                        P, fx, fy, tq, deep);
        };
        // the search only collects candidates; their forces are computed
        // afterwards, so the lanes of the warp do the costly part in step
        int nc = 0;
        short *cl = sm.clist + lane;
        auto flush = [&]() {
            for (int i = 0; i < nc; i++) touch(cl[32 * i]);
            nc = 0;
        };
        auto hit = [&](int k) {
            if (nc == MAXC) flush();
            cl[32 * nc] = (short)k;
            nc++;
        };
        auto scan = [&](int k0, int k1, float xs, float ys, bool mix, bool miy) {
            for (int k = k0; k < k1; k++) {
                const float4 q = sm.S4[k];
                float dx = q.x - xs, dy = q.y - ys;
                if (mix) dx = min_image(dx, Lx, iLx);
                if (miy) dy = min_image(dy, Ly, iLy);
                const float S = pl.z + q.z;
                if (fmaf(S, S, -(dx * dx + dy * dy)) > 0.0f && k != p) hit(k);
            }
        };
        const bool small = p < nsmall;
        if (small) {
            // 3 x 3 bins: per row at most two contiguous runs of bins (one
            // with the periodic shift), walked as one loop
            const int bx = (int)__umulhi(ql.x, (unsigned)nb), by = (int)__umulhi(ql.y, (unsigned)nb);
            int a0 = bx - 1, a1 = bx + 1, c0 = 1, c1 = 0;
            float xc = pl.x;
            if (bx == 0) { a0 = 0; a1 = 1; c0 = nb - 1; c1 = nb - 1; xc = pl.x + Lx; }
            else if (bx == nb - 1) { a0 = nb - 2; a1 = nb - 1; c0 = 0; c1 = 0; xc = pl.x - Lx; }
#pragma unroll
            for (int dyb = -1; dyb <= 1; dyb++) {
                int wy = by + dyb;
                float ys = pl.y;
                if (wy < 0) { wy += nb; ys += Ly; } else if (wy >= nb) { wy -= nb; ys -= Ly; }
                const int row = wy * nb;
                const int kA = sm.bst[row + a0], nA = sm.bst[row + a1 + 1] - kA;
                const int kC = sm.bst[row + c0], nC = c1 >= c0 ? sm.bst[row + c1 + 1] - kC : 0;
                for (int i = 0; i < nA + nC; i++) {
                    const bool inA = i < nA;
                    const int k = inA ? kA + i : kC + (i - nA);
                    const float4 q = sm.S4[k];
                    const float dx = q.x - (inA ? pl.x : xc), dy = q.y - ys;
                    const float S = pl.z + q.z;
                    if (fmaf(S, S, -(dx * dx + dy * dy)) > 0.0f && k != p) hit(k);
                }
            }
        } else if (nb) {
            // a large floe: the small floes' bins within its reach
            const float reach = 1.001f * (pl.z + Rs);
            const float rx = reach_cap(reach, Lx), ry = reach_cap(reach, Ly);
            int bx0 = (int)floorf((pl.x - rx) / Bx), bx1 = (int)floorf((pl.x + rx) / Bx);
            int by0 = (int)floorf((pl.y - ry) / By), by1 = (int)floorf((pl.y + ry) / By);
            const bool allx = bx1 - bx0 + 1 >= nb, ally = by1 - by0 + 1 >= nb;
            if (allx) { bx0 = 0; bx1 = nb - 1; }
            if (ally) { by0 = 0; by1 = nb - 1; }
            for (int by = by0; by <= by1; by++) {
                const int wy = by < 0 ? by + nb : (by >= nb ? by - nb : by);
                const float ys = ally ? pl.y : (by < 0 ? pl.y + Ly : (by >= nb ? pl.y - Ly : pl.y));
                const int row = wy * nb;
                if (allx) {
                    scan(sm.bst[row], sm.bst[row + nb], pl.x, ys, true, ally);
                } else {
                    if (bx0 < 0) scan(sm.bst[row + bx0 + nb], sm.bst[row + nb], pl.x + Lx, ys, false, ally);
                    const int a0 = bx0 < 0 ? 0 : bx0, a1 = bx1 > nb - 1 ? nb - 1 : bx1;
                    scan(sm.bst[row + a0], sm.bst[row + a1 + 1], pl.x, ys, false, ally);
                    if (bx1 >= nb) scan(sm.bst[row], sm.bst[row + bx1 - nb + 1], pl.x - Lx, ys, false, ally);
                }
            }
        }
        scan(nsmall, n, pl.x, pl.y, true, true);
        flush();

        // ---- drag, forward Euler, gradual update, moments
        const float xf = (float)ql.x * INV2_32F, yf = (float)ql.y * INV2_32F;
        float uo = P.uo_x, vo = P.uo_y, zeta = 0.0f;
        if (P.taylor) {
            for (int m = 0; m < P.n_modes; m++) {
                float c0, s0;
                rot_small(fmaf(P.ta[m], xf, P.tb[m] * yf), c0, s0);
                const float2 C = sm.Cm[m];
                const float cs = C.x * c0 - C.y * s0, sn = C.y * c0 + C.x * s0;
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        } else {
            for (int m = 0; m < P.n_modes; m++) {
                const float cyc = sm.Cm[m].x + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
                float sn, cs;
                sincospif(2.0f * cyc, &sn, &cs);
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        }
        float Fdx, Fdy, Td;
        drag_force(P, uo, vo, zeta, bs.ua, bs.va, vl.x, vl.y, vl.z, pl.z, Fdx, Fdy, Td);
        fx += Fdx; fy += Fdy; tq += Td;
        const float r = pl.z, h = pl.w;
        const float mass = P.mass_c * r * r * h;
        const float I = P.inertia_f * mass * r * r;
        float un = vl.x + dt * (fx / mass);
        float vn = vl.y + dt * (fy / mass);
        float wn = vl.z + dt * (tq / I);
        float rn = r;
        if (bs.ramp) {
            rn = r * rg;
            un += rdu;
            vn += rdv;
            wn += rdw;
        }
        bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
        const int gi = o + sm.orig[p];
        out.u[gi] = un;
        out.v[gi] = vn;
        out.w[gi] = wn;
        if (bs.ramp || out.r != in.r) out.r[gi] = rn;
        float a12[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; k++) a12[k] = 0.0f;
        add_moments(a12, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
#pragma unroll
        for (int k = 1; k < NMOM; k++) acc[k] += a12[k];
    }
    // ---- moments: lane 2k holds the warp total of column k
    const float tot = warp_sum16(acc, lane);
    const double dtot = (double)tot;
    const double M = __shfl_sync(FULL, dtot, 2), Mu = __shfl_sync(FULL, dtot, 4), Mv = __shfl_sync(FULL, dtot, 6);
    const double Fx = __shfl_sync(FULL, dtot, 18), Fy = __shfl_sync(FULL, dtot, 20), Tz = __shfl_sync(FULL, dtot, 22);
    double *mo = sc.mom + (size_t)c * NMOM;
    if ((lane & 1) == 0 && lane < 2 * NMOM) mo[lane >> 1] = lane == 0 ? (double)n : dtot;
    if (lane == 0 && sc.couple) {
        const int nc = sc.ncell;
        if (M > 0.0) {
            sc.win[c] += Mu / M;
            sc.win[nc + c] += Mv / M;
        }
        sc.win[2 * nc + c] += Fx;
        sc.win[3 * nc + c] += Fy;
        sc.win[4 * nc + c] += Tz;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&sc.ctrl->deep, 1ull);
}

// ============================================= FP32 warp, neighbour lists
// The warp kernel with per-floe contact candidate lists kept across steps
// (variant 4).  A floe moves about |v| dt per step (metres) against radii and
// bins of kilometres, so the pairs within r_l + r_j + skin found by the bin
// search stay a superset of the contacts for several steps.  A cell rebuilds
// its lists (the full binned search of k_cell_step32_warp with the reach
// widened by the skin) at the first step of every gradual-update period (its
// radii may just have changed), when any floe has moved more than half the
// skin since the build, or when a list overflowed; otherwise each floe only
// tests its list.  A floe's count and first NLH entries are one 16-byte head
// (consecutive floes' heads are adjacent, so the lanes' loads coalesce); the
// rest follow in 16-byte groups.  Contact forces are summed in list order,
// which is the search order of the build.

// Shared memory per warp: 30 B per floe (the search and the lists need the
// fixed-point position for the periodic minimum image, radius, thickness,
// velocity and spin; the angle goes from global memory to global memory).
__host__ __device__ inline size_t list_region_bytes(int cap, int nbmax)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    return a16(sizeof(float4) * cap) + a16(sizeof(uint2) * cap) + a16(sizeof(float) * cap) +
           a16(sizeof(short) * cap) + a16(sizeof(short) * MAXC * 32) + 2 * a16(sizeof(int) * (nbmax * nbmax + 1)) +
           a16(sizeof(float2) * MAXM);
}

struct ListSm {
    float4 *P4;    // r, h, u, v
    uint2 *SQ;     // exact fixed-point position
    float *W;      // spin
    short *orig;   // floe slot in the cell (search order -> slot)
    short *clist;  // [MAXC][32] contact candidates per lane
    int *cnt, *bst;
    float2 *Cm;    // per mode: (cos, sin) of the cell's phase, or (phase, -)
};

__device__ __forceinline__ ListSm carve_list(unsigned char *p, int cap, int nbmax)
{
    ListSm w;
    size_t o = 0;
    w.P4 = reinterpret_cast<float4 *>(p + o); o += align16(sizeof(float4) * cap);
    w.SQ = reinterpret_cast<uint2 *>(p + o); o += align16(sizeof(uint2) * cap);
    w.W = reinterpret_cast<float *>(p + o); o += align16(sizeof(float) * cap);
    w.orig = reinterpret_cast<short *>(p + o); o += align16(sizeof(short) * cap);
    w.clist = reinterpret_cast<short *>(p + o); o += align16(sizeof(short) * MAXC * 32);
    w.cnt = reinterpret_cast<int *>(p + o); o += align16(sizeof(int) * (nbmax * nbmax + 1));
    w.bst = reinterpret_cast<int *>(p + o); o += align16(sizeof(int) * (nbmax * nbmax + 1));
    w.Cm = reinterpret_cast<float2 *>(p + o);
    return w;
}

// a list entry's partner as the warp list kernel stages it
struct PartnerW {
    uint2 q;     // fixed-point position
    float4 p;    // r, h, u, v
    float w;     // spin
};

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 6)
k_cell_step32_wlist(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, float beta, int item0,
                    int item1, int cap, int nbmax, int seg)
{
    const NbLists &nl = sc.nl;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockStep bs;
    block_step_init(bs, sc, P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = item0 + blockIdx.x * WARPS + warp;
    if (sc.live) item1 = min(item1, item0 + sc.live[seg]);
    if (item >= item1) return;
    const ListSm sm = carve_list(smem + warp * list_region_bytes(cap, nbmax), cap, nbmax);
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;

    const float dt = sc.k.dt;
    const float Lx = sc.k.Lx, Ly = sc.k.Ly;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    const int c = sc.order[item];
    const int o = sc.off[c], n = sc.off[c + 1] - o;
    const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;
    const long long sidx = sc.ctrl->base + sc.i_local + 1;     // this step's index

    float rg = 1.0f, rdu = 0.0f, rdv = 0.0f, rdw = 0.0f;
    if (bs.ramp) {
        if (lane == 0) {
            const RampCell rc = ramp_cell(sc, c, bs.ev);
            rg = (float)rc.g; rdu = (float)rc.du; rdv = (float)rc.dv; rdw = (float)rc.dw;
        }
        rg = __shfl_sync(FULL, rg, 0); rdu = __shfl_sync(FULL, rdu, 0);
        rdv = __shfl_sync(FULL, rdv, 0); rdw = __shfl_sync(FULL, rdw, 0);
    }
    if (lane < P.n_modes) {
        const int m = lane;
        const float b = corner_phase(P, m, ix, iy, sc.g.nx, sc.g.nyr, inx, iny);
        float sn, cs;
        if (P.taylor) {
            sincospif(2.0f * b, &sn, &cs);
            sm.Cm[m] = make_float2(cs, sn);
        } else {
            sm.Cm[m] = make_float2(b, 0.0f);
        }
    }

    // ---- keep the lists or rebuild them?
    const long long built = nl.cstep[c];
    const float skin0 = nl.skin[c];
    bool rebuild = (sc.i_local % sc.n_t == 0) || built < 0 || sidx - built >= sc.n_t || sidx < built;
    uint4 hn = make_uint4(0u, 0u, 0u, 0u);     // list head of this lane's next floe
    if (!rebuild) {
        if (lane < n) hn = nl.head[o + lane];
        // the cell in floe order, and the displacement check, in one pass:
        // all of a floe's loads are independent
        const float lim = 0.25f * skin0 * skin0;
        bool far = false;
        for (int k = lane; k < n; k += 32) {
            const uint2 b = nl.xb[o + k];
            const uint32_t xq = in.xq[o + k], yq = in.yq[o + k];
            const float r = in.r[o + k], h = in.h[o + k], u = in.u[o + k], v = in.v[o + k], w = in.w[o + k];
            const float dx = (float)(int)(xq - b.x) * sx, dy = (float)(int)(yq - b.y) * sy;
            far |= dx * dx + dy * dy > lim;
            sm.P4[k] = make_float4(r, h, u, v);
            sm.W[k] = w;
            sm.SQ[k] = make_uint2(xq, yq);
        }
        rebuild = __any_sync(FULL, far);
    }

    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = 0.0f;
    unsigned deep = 0;
    bool bad = false;
    // drag, forward Euler, gradual update and moments of floe k (stored slot)
    // given its contact force; shared by both paths
    auto finish = [&](int k, const uint2 &ql, const float4 &pl, float wl, float fx, float fy, float tq) {
        const float xf = (float)ql.x * INV2_32F, yf = (float)ql.y * INV2_32F;
        float uo = P.uo_x, vo = P.uo_y, zeta = 0.0f;
        if (P.taylor) {
            for (int m = 0; m < P.n_modes; m++) {
                float c0, s0;
                rot_small(fmaf(P.ta[m], xf, P.tb[m] * yf), c0, s0);
                const float2 C = sm.Cm[m];
                const float cs = C.x * c0 - C.y * s0, sn = C.y * c0 + C.x * s0;
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        } else {
            for (int m = 0; m < P.n_modes; m++) {
                const float cyc = sm.Cm[m].x + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
                float sn, cs;
                sincospif(2.0f * cyc, &sn, &cs);
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        }
        float Fdx, Fdy, Td;
        drag_force(P, uo, vo, zeta, bs.ua, bs.va, pl.z, pl.w, wl, pl.x, Fdx, Fdy, Td);
        fx += Fdx; fy += Fdy; tq += Td;
        const float r = pl.x, h = pl.y;
        const float mass = P.mass_c * r * r * h;
        const float I = P.inertia_f * mass * r * r;
        const float dtm = dt / mass;
        float un = pl.z + dtm * fx;
        float vn = pl.w + dtm * fy;
        float wn = wl + dt * (tq / I);
        float rn = r;
        if (bs.ramp) {
            rn = r * rg;
            un += rdu;
            vn += rdv;
            wn += rdw;
        }
        bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
        const int gi = o + k;
        out.u[gi] = un;
        out.v[gi] = vn;
        out.w[gi] = wn;
        if (bs.ramp || out.r != in.r) out.r[gi] = rn;
        float a12[NMOM];
#pragma unroll
        for (int q = 0; q < NMOM; q++) a12[q] = 0.0f;
        add_moments(a12, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
#pragma unroll
        for (int q = 1; q < NMOM; q++) acc[q] += a12[q];
    };

    if (!rebuild) {
        // ---- each floe tests its list (the next floe's head is loaded while
        // this floe's candidates are tested)
        __syncwarp();
        for (int p = lane; p < n; p += 32) {
            const uint4 hd = hn;
            if (p + 32 < n) hn = nl.head[o + p + 32];
            const float4 pl = sm.P4[p];
            const float wl = sm.W[p];
            const uint2 ql = sm.SQ[p];
            out.xq[o + p] = ql.x + (uint32_t)__float2int_rn(dt * pl.z * isx);
            out.yq[o + p] = ql.y + (uint32_t)__float2int_rn(dt * pl.w * isy);
            out.th[o + p] = in.th[o + p] + dt * wl;
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            list_walk(
                hd, nl.tail + (size_t)(o + p) * NLT, [&](int j) { return PartnerW{sm.SQ[j], sm.P4[j], sm.W[j]}; },
                [&](const PartnerW &b) {
                    const float dx = (float)(int)(b.q.x - ql.x) * sx;
                    const float dy = (float)(int)(b.q.y - ql.y) * sy;
                    contact_add(dx, dy, dx * dx + dy * dy, pl.x, b.p.x, pl.y, b.p.y, b.p.z - pl.z, b.p.w - pl.w, wl,
                                b.w, P, fx, fy, tq, deep);
                });
            finish(p, ql, pl, wl, fx, fy, tq);
        }
    } else {
        // ---- rebuild: the binned search of k_cell_step32_warp with the reach
        // widened by the skin, recording every candidate
        float vmax = 0.0f;
        for (int k = lane; k < n; k += 32) vmax = fmaxf(vmax, fmaxf(fabsf(in.u[o + k]), fabsf(in.v[o + k])));
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(FULL, vmax, d));
        // over one gradual-update period a floe moving at the cell's largest
        // speed covers 0.71 of half the skin (sqrt 2 for both axes)
        const float skin = 4.0f * vmax * dt * (float)sc.n_t + 1.0e-3f;
        int nb = (int)(sqrtf((float)n) / beta);
        nb = nb > nbmax ? nbmax : nb;
        if (nb < 3) nb = 0;
        const float Bx = nb ? Lx / nb : Lx, By = nb ? Ly / nb : Ly;
        const float Rs = nb ? 0.5f * fminf(Bx, By) - 0.5f * skin : -1.0f;
        const int nbins = nb * nb;
        for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
        __syncwarp();
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < n;
            const uint32_t xq = valid ? in.xq[o + k] : 0u, yq = valid ? in.yq[o + k] : 0u;
            const float r = valid ? in.r[o + k] : 0.0f;
            const bool small = valid && r <= Rs;
            const int b = small ? (int)(__umulhi(yq, (unsigned)nb) * nb + __umulhi(xq, (unsigned)nb)) : -1 - lane;
            const unsigned m = __match_any_sync(FULL, b);
            if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
            __syncwarp();
        }
        const int nsmall = warp_scan_excl(sm.cnt, sm.bst, nbins + 1, lane);
        for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
        __syncwarp();
        int lrun = nsmall;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < n;
            uint32_t xq = 0u, yq = 0u;
            float r = 0.0f, h = 0.0f, u = 0.0f, v = 0.0f, w = 0.0f, th = 0.0f;
            if (valid) {
                xq = in.xq[o + k]; yq = in.yq[o + k];
                r = in.r[o + k]; h = in.h[o + k];
                u = in.u[o + k]; v = in.v[o + k]; w = in.w[o + k]; th = in.th[o + k];
            }
            const bool small = valid && r <= Rs;
            const bool large = valid && !small;
            const int b = small ? (int)(__umulhi(yq, (unsigned)nb) * nb + __umulhi(xq, (unsigned)nb)) : -1 - lane;
            const unsigned m = __match_any_sync(FULL, b);
            const unsigned bl = __ballot_sync(FULL, large);
            int pos = 0;
            if (small) pos = sm.bst[b] + sm.cnt[b] + __popc(m & lt);
            else if (large) pos = lrun + __popc(bl & lt);
            if (valid) {
                sm.P4[pos] = make_float4(r, h, u, v);
                sm.W[pos] = w;
                sm.SQ[pos] = make_uint2(xq, yq);
                sm.orig[pos] = (short)k;
                out.xq[o + k] = xq + (uint32_t)__float2int_rn(dt * u * isx);
                out.yq[o + k] = yq + (uint32_t)__float2int_rn(dt * v * isy);
                out.th[o + k] = th + dt * w;
                nl.xb[o + k] = make_uint2(xq, yq);
            }
            __syncwarp();
            if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
            lrun += __popc(bl);
            __syncwarp();
        }
        bool overflow = false;
        for (int p = lane; p < n; p += 32) {
            const float4 pl = sm.P4[p];
            const float wl = sm.W[p];
            const uint2 ql = sm.SQ[p];
            const int kp = sm.orig[p];
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            ListRec rec;
            uint16_t *tail16 = reinterpret_cast<uint16_t *>(nl.tail + (size_t)(o + kp) * NLT);
            auto touch = [&](int k) {
                const uint2 qj = sm.SQ[k];
                const float dx = (float)(int)(qj.x - ql.x) * sx;
                const float dy = (float)(int)(qj.y - ql.y) * sy;
                const float4 pj = sm.P4[k];
                contact_add(dx, dy, dx * dx + dy * dy, pl.x, pj.x, pl.y, pj.y, pj.z - pl.z, pj.w - pl.w, wl,
                            sm.W[k], P, fx, fy, tq, deep);
                rec.add(tail16, sm.orig[k]);
            };
            int ncand = 0;
            short *cl = sm.clist + lane;
            auto flush = [&]() {
                for (int i = 0; i < ncand; i++) touch(cl[32 * i]);
                ncand = 0;
            };
            auto hit = [&](int k) {
                if (ncand == MAXC) flush();
                cl[32 * ncand] = (short)k;
                ncand++;
            };
            // candidate test: the 32-bit fixed-point difference is the
            // periodic minimum image in the cell, whichever bin k came from
            auto test = [&](int k) {
                const uint2 qk = sm.SQ[k];
                const float dx = (float)(int)(qk.x - ql.x) * sx, dy = (float)(int)(qk.y - ql.y) * sy;
                const float S = pl.x + sm.P4[k].x + skin;
                if (fmaf(S, S, -(dx * dx + dy * dy)) > 0.0f && k != p) hit(k);
            };
            auto scan = [&](int k0, int k1) {
                for (int k = k0; k < k1; k++) test(k);
            };
            const bool small = p < nsmall;
            if (small) {
                const int bx = (int)__umulhi(ql.x, (unsigned)nb), by = (int)__umulhi(ql.y, (unsigned)nb);
                int a0 = bx - 1, a1 = bx + 1, c0 = 1, c1 = 0;
                if (bx == 0) { a0 = 0; a1 = 1; c0 = nb - 1; c1 = nb - 1; }
                else if (bx == nb - 1) { a0 = nb - 2; a1 = nb - 1; c0 = 0; c1 = 0; }
#pragma unroll
                for (int dyb = -1; dyb <= 1; dyb++) {
                    int wy = by + dyb;
                    if (wy < 0) wy += nb; else if (wy >= nb) wy -= nb;
                    const int row = wy * nb;
                    const int kA = sm.bst[row + a0], nA = sm.bst[row + a1 + 1] - kA;
                    const int kC = sm.bst[row + c0], nC = c1 >= c0 ? sm.bst[row + c1 + 1] - kC : 0;
                    for (int i = 0; i < nA + nC; i++) test(i < nA ? kA + i : kC + (i - nA));
                }
            } else if (nb) {
                const float xl = (float)ql.x * sx, yl = (float)ql.y * sy;
                const float reach = 1.001f * (pl.x + Rs + skin);
                const float rx = reach_cap(reach, Lx), ry = reach_cap(reach, Ly);
                int bx0 = (int)floorf((xl - rx) / Bx), bx1 = (int)floorf((xl + rx) / Bx);
                int by0 = (int)floorf((yl - ry) / By), by1 = (int)floorf((yl + ry) / By);
                const bool allx = bx1 - bx0 + 1 >= nb, ally = by1 - by0 + 1 >= nb;
                if (allx) { bx0 = 0; bx1 = nb - 1; }
                if (ally) { by0 = 0; by1 = nb - 1; }
                for (int by = by0; by <= by1; by++) {
                    const int wy = by < 0 ? by + nb : (by >= nb ? by - nb : by);
                    const int row = wy * nb;
                    if (allx) {
                        scan(sm.bst[row], sm.bst[row + nb]);
                    } else {
                        if (bx0 < 0) scan(sm.bst[row + bx0 + nb], sm.bst[row + nb]);
                        const int a0 = bx0 < 0 ? 0 : bx0, a1 = bx1 > nb - 1 ? nb - 1 : bx1;
                        scan(sm.bst[row + a0], sm.bst[row + a1 + 1]);
                        if (bx1 >= nb) scan(sm.bst[row], sm.bst[row + bx1 - nb + 1]);
                    }
                }
            }
            scan(nsmall, n);
            flush();
            overflow |= rec.nlst > NBL;
            nl.head[o + kp] = rec.head();
            finish(kp, ql, pl, wl, fx, fy, tq);
        }
        const bool any_over = __any_sync(FULL, overflow);
        if (lane == 0) {
            nl.cstep[c] = any_over ? -1 : sidx;     // an overflowing cell searches again next step
            nl.skin[c] = skin;
        }
    }

    // ---- moments: lane 2k holds the warp total of column k
    const float tot = warp_sum16(acc, lane);
    const double dtot = (double)tot;
    const double M = __shfl_sync(FULL, dtot, 2), Mu = __shfl_sync(FULL, dtot, 4), Mv = __shfl_sync(FULL, dtot, 6);
    const double Fx = __shfl_sync(FULL, dtot, 18), Fy = __shfl_sync(FULL, dtot, 20), Tz = __shfl_sync(FULL, dtot, 22);
    double *mo = sc.mom + (size_t)c * NMOM;
    if ((lane & 1) == 0 && lane < 2 * NMOM) mo[lane >> 1] = lane == 0 ? (double)n : dtot;
    if (lane == 0 && sc.couple) {
        const int nc = sc.ncell;
        if (M > 0.0) {
            sc.win[c] += Mu / M;
            sc.win[nc + c] += Mv / M;
        }
        sc.win[2 * nc + c] += Fx;
        sc.win[3 * nc + c] += Fy;
        sc.win[4 * nc + c] += Tz;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&sc.ctrl->deep, 1ull);
}

// ======================================================= FP32 warp, resident
// The warp kernel's step, repeated for a run of fine steps with the cell kept
// in shared memory.  Between coarse steps a cell depends on nothing but
// itself (its gradual-update increments are fixed at the coarse step), so a
// warp can take its cell through a whole coarse interval and touch global
// memory only at the two ends.  Every step is written as the step of
// k_cell_step32_warp (same search order, same sums; the compiler may still
// fuse a multiply-add differently in the two kernels), and a run of steps
// gives the floes, moments and window of the same number of one-step
// launches of this kernel, bit for bit.
//
// Shared memory per warp: the cell in floe order (home: position, velocity,
// spin, radius, angle, thickness), updated in place at the end of each step,
// and the search-order copy of the step's start state that the contact
// search reads.

__host__ __device__ inline size_t run_region_bytes(int cap, int nbmax)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    return a16(sizeof(uint2) * cap) + a16(sizeof(float4) * cap) + a16(sizeof(float2) * cap) +
           warp_region_bytes(cap, nbmax) + a16(sizeof(double) * NWIN);
}

struct RunSm {
    uint2 *HQ;     // home: fixed-point position
    float4 *HU;    // home: u, v, w, r
    float2 *HT;    // home: theta, h
    double *win;   // the cell's window sums over the run
    WarpSm w;      // search-order copy and bins, as in the single-step kernel
};

__device__ __forceinline__ RunSm carve_run(unsigned char *p, int cap, int nbmax)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    RunSm r;
    size_t o = 0;
    r.HQ = reinterpret_cast<uint2 *>(p + o); o += a16(sizeof(uint2) * cap);
    r.HU = reinterpret_cast<float4 *>(p + o); o += a16(sizeof(float4) * cap);
    r.HT = reinterpret_cast<float2 *>(p + o); o += a16(sizeof(float2) * cap);
    r.win = reinterpret_cast<double *>(p + o); o += a16(sizeof(double) * NWIN);
    r.w = carve_warp(p + o, cap, nbmax);
    return r;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 5)
k_cell_run32_warp(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, int nsteps, float beta, int item0,
                  int item1, int cap, int nbmax, int seg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = item0 + blockIdx.x * WARPS + warp;
    if (sc.live) item1 = min(item1, item0 + sc.live[seg]);
    if (item >= item1) return;
    const RunSm R = carve_run(smem + warp * run_region_bytes(cap, nbmax), cap, nbmax);
    const WarpSm &sm = R.w;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;

    const float dt = sc.k.dt;
    const float Lx = sc.k.Lx, Ly = sc.k.Ly, iLx = sc.k.iLx, iLy = sc.k.iLy;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    const int c = sc.order[item];
    const int o = sc.off[c], n = sc.off[c + 1] - o;
    const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;
    const long long base = sc.ctrl->base;
    const bool have_tgt = sc.couple && sc.ctrl->have_tgt;
    const int nc = sc.ncell;

    // ---- the cell into shared memory; window sums so far
    for (int k = lane; k < n; k += 32) {
        R.HQ[k] = make_uint2(in.xq[o + k], in.yq[o + k]);
        R.HU[k] = make_float4(in.u[o + k], in.v[o + k], in.w[o + k], in.r[o + k]);
        R.HT[k] = make_float2(in.th[o + k], in.h[o + k]);
    }
    if (sc.couple && lane < NWIN) R.win[lane] = sc.win[(size_t)lane * nc + c];
    if (lane < P.n_modes) {
        const int m = lane;
        const float b = corner_phase(P, m, ix, iy, sc.g.nx, sc.g.nyr, inx, iny);
        float sn, cs;
        if (P.taylor) {
            sincospif(2.0f * b, &sn, &cs);
            sm.Cm[m] = make_float2(cs, sn);
        } else {
            sm.Cm[m] = make_float2(b, 0.0f);
        }
    }
    int nb = (int)(sqrtf((float)n) / beta);
    nb = nb > nbmax ? nbmax : nb;
    if (nb < 3) nb = 0;
    const float Bx = nb ? Lx / nb : Lx, By = nb ? Ly / nb : Ly;
    const float Rs = nb ? 0.5f * fminf(Bx, By) : -1.0f;
    const int nbins = nb * nb;
    __syncwarp();

    unsigned deep_steps = 0;
    bool bad = false;
    float wua = 0.0f, wva = 0.0f;     // lane i: wind of step j0 + 32 q + i
    const int j0 = (int)sc.i_local;
    for (int js = 0; js < nsteps; js++) {
        const int j = j0 + js;
        // wind at the start of each step, 32 steps at a time (one FP64
        // evaluation per lane)
        if ((js & 31) == 0) {
            const long long sj = base + j + lane + 1;
            wind_at(P, (double)(sj - 1) * sc.dt, wua, wva);
        }
        const float ua = __shfl_sync(FULL, wua, js & 31), va = __shfl_sync(FULL, wva, js & 31);
        const long long kk = (long long)j + 1;
        const bool ramp = have_tgt && (kk % sc.n_t == 0);
        float rg = 1.0f, rdu = 0.0f, rdv = 0.0f, rdw = 0.0f;
        if (ramp) {
            if (lane == 0) {
                const RampCell rc = ramp_cell(sc, c, (int)(kk / sc.n_t));
                rg = (float)rc.g; rdu = (float)rc.du; rdv = (float)rc.dv; rdw = (float)rc.dw;
            }
            rg = __shfl_sync(FULL, rg, 0); rdu = __shfl_sync(FULL, rdu, 0);
            rdv = __shfl_sync(FULL, rdv, 0); rdw = __shfl_sync(FULL, rdw, 0);
        }

        for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
        __syncwarp();
        // ---- count small floes per bin
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < n;
            const uint2 q = valid ? R.HQ[k] : make_uint2(0u, 0u);
            const float r = valid ? R.HU[k].w : 0.0f;
            const bool small = valid && r <= Rs;
            const int b = small ? (int)(__umulhi(q.y, (unsigned)nb) * nb + __umulhi(q.x, (unsigned)nb)) : -1 - lane;
            const unsigned m = __match_any_sync(FULL, b);
            if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
            __syncwarp();
        }
        const int nsmall = warp_scan_excl(sm.cnt, sm.bst, nbins + 1, lane);
        for (int b = lane; b <= nbins; b += 32) sm.cnt[b] = 0;
        __syncwarp();
        // ---- place every floe at its search position; position and angle
        // advance at once (they need only the floe's own start state)
        int lrun = nsmall;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < n;
            uint2 q = make_uint2(0u, 0u);
            float4 U = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float2 T = make_float2(0.0f, 0.0f);
            if (valid) {
                q = R.HQ[k];
                U = R.HU[k];
                T = R.HT[k];
            }
            const float r = U.w;
            const bool small = valid && r <= Rs;
            const bool large = valid && !small;
            const int b = small ? (int)(__umulhi(q.y, (unsigned)nb) * nb + __umulhi(q.x, (unsigned)nb)) : -1 - lane;
            const unsigned m = __match_any_sync(FULL, b);
            const unsigned bl = __ballot_sync(FULL, large);
            int pos = 0;
            if (small) pos = sm.bst[b] + sm.cnt[b] + __popc(m & lt);
            else if (large) pos = lrun + __popc(bl & lt);
            if (valid) {
                sm.S4[pos] = make_float4((float)q.x * sx, (float)q.y * sy, r, T.y);
                sm.SV[pos] = make_float4(U.x, U.y, U.z, 0.0f);
                sm.SQ[pos] = q;
                sm.orig[pos] = (short)k;
                R.HQ[k] = make_uint2(q.x + (uint32_t)__float2int_rn(dt * U.x * isx),
                                     q.y + (uint32_t)__float2int_rn(dt * U.y * isy));
                R.HT[k].x = T.x + dt * U.z;
            }
            __syncwarp();
            if (small && lane == __ffs(m) - 1) sm.cnt[b] += __popc(m);
            lrun += __popc(bl);
            __syncwarp();
        }

        float acc[16];
#pragma unroll
        for (int k = 0; k < 16; k++) acc[k] = 0.0f;
        unsigned deep = 0;
        for (int p = lane; p < n; p += 32) {
            const float4 pl = sm.S4[p];
            const float4 vl = sm.SV[p];
            const uint2 ql = sm.SQ[p];
            float fx = 0.0f, fy = 0.0f, tq = 0.0f;
            auto touch = [&](int k) {
                const uint2 qj = sm.SQ[k];
                const float dx = (float)(int)(qj.x - ql.x) * sx;
                const float dy = (float)(int)(qj.y - ql.y) * sy;
                const float4 pj = sm.S4[k];
                const float4 vj = sm.SV[k];
                contact_add(dx, dy, dx * dx + dy * dy, pl.z, pj.z, pl.w, pj.w, vj.x - vl.x, vj.y - vl.y, vl.z,
                            vj.z, P, fx, fy, tq, deep);
            };
            int ncand = 0;
            short *cl = sm.clist + lane;
            auto flush = [&]() {
                for (int i = 0; i < ncand; i++) touch(cl[32 * i]);
                ncand = 0;
            };
            auto hit = [&](int k) {
                if (ncand == MAXC) flush();
                cl[32 * ncand] = (short)k;
                ncand++;
            };
            auto scan = [&](int k0, int k1, float xs, float ys, bool mix, bool miy) {
                for (int k = k0; k < k1; k++) {
                    const float4 q = sm.S4[k];
                    float dx = q.x - xs, dy = q.y - ys;
                    if (mix) dx = min_image(dx, Lx, iLx);
                    if (miy) dy = min_image(dy, Ly, iLy);
                    const float S = pl.z + q.z;
                    if (fmaf(S, S, -(dx * dx + dy * dy)) > 0.0f && k != p) hit(k);
                }
            };
            const bool small = p < nsmall;
            if (small) {
                const int bx = (int)__umulhi(ql.x, (unsigned)nb), by = (int)__umulhi(ql.y, (unsigned)nb);
                int a0 = bx - 1, a1 = bx + 1, c0 = 1, c1 = 0;
                float xc = pl.x;
                if (bx == 0) { a0 = 0; a1 = 1; c0 = nb - 1; c1 = nb - 1; xc = pl.x + Lx; }
                else if (bx == nb - 1) { a0 = nb - 2; a1 = nb - 1; c0 = 0; c1 = 0; xc = pl.x - Lx; }
#pragma unroll
                for (int dyb = -1; dyb <= 1; dyb++) {
                    int wy = by + dyb;
                    float ys = pl.y;
                    if (wy < 0) { wy += nb; ys += Ly; } else if (wy >= nb) { wy -= nb; ys -= Ly; }
                    const int row = wy * nb;
                    const int kA = sm.bst[row + a0], nA = sm.bst[row + a1 + 1] - kA;
                    const int kC = sm.bst[row + c0], nC = c1 >= c0 ? sm.bst[row + c1 + 1] - kC : 0;
                    for (int i = 0; i < nA + nC; i++) {
                        const bool inA = i < nA;
                        const int k = inA ? kA + i : kC + (i - nA);
                        const float4 q = sm.S4[k];
                        const float dx = q.x - (inA ? pl.x : xc), dy = q.y - ys;
                        const float S = pl.z + q.z;
                        if (fmaf(S, S, -(dx * dx + dy * dy)) > 0.0f && k != p) hit(k);
                    }
                }
            } else if (nb) {
                const float reach = 1.001f * (pl.z + Rs);
                const float rx = reach_cap(reach, Lx), ry = reach_cap(reach, Ly);
                int bx0 = (int)floorf((pl.x - rx) / Bx), bx1 = (int)floorf((pl.x + rx) / Bx);
                int by0 = (int)floorf((pl.y - ry) / By), by1 = (int)floorf((pl.y + ry) / By);
                const bool allx = bx1 - bx0 + 1 >= nb, ally = by1 - by0 + 1 >= nb;
                if (allx) { bx0 = 0; bx1 = nb - 1; }
                if (ally) { by0 = 0; by1 = nb - 1; }
                for (int by = by0; by <= by1; by++) {
                    const int wy = by < 0 ? by + nb : (by >= nb ? by - nb : by);
                    const float ys = ally ? pl.y : (by < 0 ? pl.y + Ly : (by >= nb ? pl.y - Ly : pl.y));
                    const int row = wy * nb;
                    if (allx) {
                        scan(sm.bst[row], sm.bst[row + nb], pl.x, ys, true, ally);
                    } else {
                        if (bx0 < 0) scan(sm.bst[row + bx0 + nb], sm.bst[row + nb], pl.x + Lx, ys, false, ally);
                        const int a0 = bx0 < 0 ? 0 : bx0, a1 = bx1 > nb - 1 ? nb - 1 : bx1;
                        scan(sm.bst[row + a0], sm.bst[row + a1 + 1], pl.x, ys, false, ally);
                        if (bx1 >= nb) scan(sm.bst[row], sm.bst[row + bx1 - nb + 1], pl.x - Lx, ys, false, ally);
                    }
                }
            }
            scan(nsmall, n, pl.x, pl.y, true, true);
            flush();

            // ---- drag, forward Euler, gradual update, moments
            const float xf = (float)ql.x * INV2_32F, yf = (float)ql.y * INV2_32F;
            float uo = P.uo_x, vo = P.uo_y, zeta = 0.0f;
            if (P.taylor) {
                for (int m = 0; m < P.n_modes; m++) {
                    float c0, s0;
                    rot_small(fmaf(P.ta[m], xf, P.tb[m] * yf), c0, s0);
                    const float2 C = sm.Cm[m];
                    const float cs = C.x * c0 - C.y * s0, sn = C.y * c0 + C.x * s0;
                    uo -= P.mAu[m] * cs;
                    vo += P.mAv[m] * cs;
                    zeta -= P.mAz[m] * sn;
                }
            } else {
                for (int m = 0; m < P.n_modes; m++) {
                    const float cyc = sm.Cm[m].x + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
                    float sn, cs;
                    sincospif(2.0f * cyc, &sn, &cs);
                    uo -= P.mAu[m] * cs;
                    vo += P.mAv[m] * cs;
                    zeta -= P.mAz[m] * sn;
                }
            }
            float Fdx, Fdy, Td;
            drag_force(P, uo, vo, zeta, ua, va, vl.x, vl.y, vl.z, pl.z, Fdx, Fdy, Td);
            fx += Fdx; fy += Fdy; tq += Td;
            const float r = pl.z, h = pl.w;
            const float mass = P.mass_c * r * r * h;
            const float I = P.inertia_f * mass * r * r;
            float un = vl.x + dt * (fx / mass);
            float vn = vl.y + dt * (fy / mass);
            float wn = vl.z + dt * (tq / I);
            float rn = r;
            if (ramp) {
                rn = r * rg;
                un += rdu;
                vn += rdv;
                wn += rdw;
            }
            bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
            R.HU[sm.orig[p]] = make_float4(un, vn, wn, rn);
            float a12[NMOM];
#pragma unroll
            for (int k = 0; k < NMOM; k++) a12[k] = 0.0f;
            add_moments(a12, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
#pragma unroll
            for (int k = 1; k < NMOM; k++) acc[k] += a12[k];
        }
        deep_steps += deep ? 1u : 0u;
        // ---- moments of the step: lane 2k holds the warp total of column k
        const float tot = warp_sum16(acc, lane);
        const double dtot = (double)tot;
        const double M = __shfl_sync(FULL, dtot, 2), Mu = __shfl_sync(FULL, dtot, 4), Mv = __shfl_sync(FULL, dtot, 6);
        const double Fx = __shfl_sync(FULL, dtot, 18), Fy = __shfl_sync(FULL, dtot, 20), Tz = __shfl_sync(FULL, dtot, 22);
        if (js == nsteps - 1) {
            double *mo = sc.mom + (size_t)c * NMOM;
            if ((lane & 1) == 0 && lane < 2 * NMOM) mo[lane >> 1] = lane == 0 ? (double)n : dtot;
        }
        if (lane == 0 && sc.couple) {
            if (M > 0.0) {
                R.win[0] += Mu / M;
                R.win[1] += Mv / M;
            }
            R.win[2] += Fx;
            R.win[3] += Fy;
            R.win[4] += Tz;
        }
        __syncwarp();
    }

    // ---- the cell back to global memory
    for (int k = lane; k < n; k += 32) {
        const uint2 q = R.HQ[k];
        const float4 U = R.HU[k];
        out.xq[o + k] = q.x;
        out.yq[o + k] = q.y;
        out.th[o + k] = R.HT[k].x;
        out.u[o + k] = U.x;
        out.v[o + k] = U.y;
        out.w[o + k] = U.z;
        out.r[o + k] = U.w;
    }
    if (sc.couple && lane < NWIN) sc.win[(size_t)lane * nc + c] = R.win[lane];
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep_steps) atomicAdd(&sc.ctrl->deep, (unsigned long long)deep_steps);
}

// ================================================= FP32 packed warps, resident
// Cells of at most 32 floes (few-floe cells, as in an ensemble of sparse
// realizations), several to a warp with a lane per floe: the lanes of one
// cell are contiguous, and a host table lists each warp's cells (consecutive
// in the processing order, 32 floes at most together).  Each lane keeps its
// floe in registers for the whole run of steps; shared memory holds only the
// copy of the step's start state that the other lanes of the cell read.  No
// bins: a lane tests every other floe of its cell, in floe order.  A cell's
// moments are a segmented shuffle sum over its lanes (a fixed tree order).

constexpr int PACKW = 32;   // floes (and cells) per packed warp at most

struct PackSm {
    uint2 *Q;      // [32] fixed-point position
    float4 *A;     // [32] u, v, w, r
    float *H;      // [32] thickness
    int *cstart, *cnum, *ccell, *coff;   // [32] the warp's cells: first lane, floes, cell, first floe
    unsigned char *slot;                 // [32] lane -> cell of the warp
    float2 *Cm;    // [32][MAXM] per cell and mode: (cos, sin) of the corner phase, or (phase, -)
};

__host__ __device__ inline size_t pack_region_bytes()
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    return a16(sizeof(uint2) * PACKW) + a16(sizeof(float4) * PACKW) + a16(sizeof(float) * PACKW) +
           4 * a16(sizeof(int) * PACKW) + a16(PACKW) + a16(sizeof(float2) * PACKW * MAXM);
}

__device__ __forceinline__ PackSm carve_pack(unsigned char *p)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    PackSm S;
    size_t o = 0;
    S.Q = reinterpret_cast<uint2 *>(p + o); o += a16(sizeof(uint2) * PACKW);
    S.A = reinterpret_cast<float4 *>(p + o); o += a16(sizeof(float4) * PACKW);
    S.H = reinterpret_cast<float *>(p + o); o += a16(sizeof(float) * PACKW);
    S.cstart = reinterpret_cast<int *>(p + o); o += a16(sizeof(int) * PACKW);
    S.cnum = reinterpret_cast<int *>(p + o); o += a16(sizeof(int) * PACKW);
    S.ccell = reinterpret_cast<int *>(p + o); o += a16(sizeof(int) * PACKW);
    S.coff = reinterpret_cast<int *>(p + o); o += a16(sizeof(int) * PACKW);
    S.slot = p + o; o += a16(PACKW);
    S.Cm = reinterpret_cast<float2 *>(p + o);
    return S;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 8)
k_cell_run32_packed(DevState32 in, DevState32 out, Phys<float> P, StepCommon sc, const int2 *pack, int npack,
                    int nsteps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wi = blockIdx.x * WARPS + warp;
    if (wi >= npack) return;
    const PackSm S = carve_pack(smem + warp * pack_region_bytes());
    const unsigned FULL = 0xffffffffu;
    const float dt = sc.k.dt;
    const float sx = sc.k.sx, sy = sc.k.sy, isx = sc.k.isx, isy = sc.k.isy, inx = sc.k.inx, iny = sc.k.iny;
    const long long base = sc.ctrl->base;
    const bool have_tgt = sc.couple && sc.ctrl->have_tgt;
    const int nc = sc.ncell;

    // ---- the warp's cells (lane j describes cell j); closure cells take no lanes
    const int2 pk = pack[wi];
    int cj = -1, oj = 0, nj = 0;
    if (lane < pk.y) {
        cj = sc.order0[pk.x + lane];
        oj = sc.off[cj];
        nj = sc.off[cj + 1] - oj;
        if (sc.skip && sc.skip[cj]) cj = -1;
        if (cj < 0) nj = 0;
    }
    int incl = nj;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (lane < pk.y) {
        S.cstart[lane] = incl - nj;
        S.cnum[lane] = nj;
        S.ccell[lane] = cj;
        S.coff[lane] = oj;
        for (int k = incl - nj; k < incl; k++) S.slot[k] = (unsigned char)lane;
    }
    __syncwarp();
    for (int idx = lane; idx < pk.y * P.n_modes; idx += 32) {
        const int j = idx / P.n_modes, m = idx - j * P.n_modes;
        const int c = S.ccell[j];
        if (c < 0) continue;
        const float b = corner_phase(P, m, c % sc.g.nx, (c / sc.g.nx) % sc.g.nyr, sc.g.nx, sc.g.nyr, inx, iny);
        float sn, cs;
        if (P.taylor) {
            sincospif(2.0f * b, &sn, &cs);
            S.Cm[j * MAXM + m] = make_float2(cs, sn);
        } else {
            S.Cm[j * MAXM + m] = make_float2(b, 0.0f);
        }
    }

    // ---- this lane's floe, kept in registers for the run
    const bool act = lane < total;
    const int j = act ? S.slot[lane] : 0;
    const int s0 = act ? S.cstart[j] : lane, n = act ? S.cnum[j] : 1;
    const int c = act ? S.ccell[j] : -1;
    const int gi = act ? S.coff[j] + (lane - s0) : 0;
    const bool head = act && lane == s0;
    uint32_t xq = 0u, yq = 0u;
    float th = 0.0f, u = 0.0f, v = 0.0f, w = 0.0f, r = 0.0f, h = 0.0f;
    if (act) {
        xq = in.xq[gi]; yq = in.yq[gi]; th = in.th[gi];
        u = in.u[gi]; v = in.v[gi]; w = in.w[gi]; r = in.r[gi]; h = in.h[gi];
    }
    double win[NWIN] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (head && sc.couple)
        for (int k = 0; k < NWIN; k++) win[k] = sc.win[(size_t)k * nc + c];

    unsigned deep_steps = 0;
    bool bad = false;
    float wua = 0.0f, wva = 0.0f;
    float acc[NMOM];
    const int j0 = (int)sc.i_local;
    for (int js = 0; js < nsteps; js++) {
        const int jstep = j0 + js;
        if ((js & 31) == 0) {
            const long long sj = base + jstep + lane + 1;
            wind_at(P, (double)(sj - 1) * sc.dt, wua, wva);
        }
        const float ua = __shfl_sync(FULL, wua, js & 31), va = __shfl_sync(FULL, wva, js & 31);
        const long long kk = (long long)jstep + 1;
        const bool ramp = have_tgt && (kk % sc.n_t == 0);
        float rg = 1.0f, rdu = 0.0f, rdv = 0.0f, rdw = 0.0f;
        if (ramp) {
            if (head) {
                const RampCell rc = ramp_cell(sc, c, (int)(kk / sc.n_t));
                rg = (float)rc.g; rdu = (float)rc.du; rdv = (float)rc.dv; rdw = (float)rc.dw;
            }
            rg = __shfl_sync(FULL, rg, s0); rdu = __shfl_sync(FULL, rdu, s0);
            rdv = __shfl_sync(FULL, rdv, s0); rdw = __shfl_sync(FULL, rdw, s0);
        }
        // start state for the other lanes of the cell
        S.Q[lane] = make_uint2(xq, yq);
        S.A[lane] = make_float4(u, v, w, r);
        S.H[lane] = h;
        __syncwarp();
        // ---- contacts with the other floes of the cell, in floe order
        float fx = 0.0f, fy = 0.0f, tq = 0.0f;
        unsigned deep = 0;
        if (act) {
            for (int k = s0; k < s0 + n; k++) {
                if (k == lane) continue;
                const uint2 qk = S.Q[k];
                const float dx = (float)(int)(qk.x - xq) * sx;
                const float dy = (float)(int)(qk.y - yq) * sy;
                const float4 ak = S.A[k];
                contact_add(dx, dy, dx * dx + dy * dy, r, ak.w, h, S.H[k], ak.x - u, ak.y - v, w, ak.z, P, fx, fy,
                            tq, deep);
            }
        }
        // ---- drag, forward Euler, gradual update
        const float xf = (float)xq * INV2_32F, yf = (float)yq * INV2_32F;
        float uo = P.uo_x, vo = P.uo_y, zeta = 0.0f;
        if (P.taylor) {
            for (int m = 0; m < P.n_modes; m++) {
                float c0, s0m;
                rot_small(fmaf(P.ta[m], xf, P.tb[m] * yf), c0, s0m);
                const float2 C = S.Cm[j * MAXM + m];
                const float cs = C.x * c0 - C.y * s0m, sn = C.y * c0 + C.x * s0m;
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        } else {
            for (int m = 0; m < P.n_modes; m++) {
                const float cyc = S.Cm[j * MAXM + m].x + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
                float sn, cs;
                sincospif(2.0f * cyc, &sn, &cs);
                uo -= P.mAu[m] * cs;
                vo += P.mAv[m] * cs;
                zeta -= P.mAz[m] * sn;
            }
        }
        float Fdx, Fdy, Td;
        drag_force(P, uo, vo, zeta, ua, va, u, v, w, r, Fdx, Fdy, Td);
        fx += Fdx; fy += Fdy; tq += Td;
        const float mass = P.mass_c * r * r * h;
        const float I = P.inertia_f * mass * r * r;
        const uint32_t xn = xq + (uint32_t)__float2int_rn(dt * u * isx);
        const uint32_t yn = yq + (uint32_t)__float2int_rn(dt * v * isy);
        const float thn = th + dt * w;
        float un = u + dt * (fx / mass);
        float vn = v + dt * (fy / mass);
        float wn = w + dt * (tq / I);
        float rn = r;
        if (ramp) {
            rn = r * rg;
            un += rdu;
            vn += rdv;
            wn += rdw;
        }
        if (act) {
            bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
            xq = xn; yq = yn; th = thn; u = un; v = vn; w = wn; r = rn;
        }
        deep_steps += deep ? 1u : 0u;
        // ---- the cell's moments: segmented sums over its lanes
#pragma unroll
        for (int k = 0; k < NMOM; k++) acc[k] = 0.0f;
        if (act) add_moments(acc, P.mass_c, P.inertia_f, un, vn, wn, rn, h, Fdx, Fdy, Td);
        const int end = s0 + n;
#pragma unroll
        for (int k = 1; k < NMOM; k++) {
            float x = acc[k];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const float y = __shfl_down_sync(FULL, x, d);
                if (lane + d < end) x += y;
            }
            acc[k] = x;
        }
        if (head) {
            if (js == nsteps - 1) {
                double *mo = sc.mom + (size_t)c * NMOM;
                mo[0] = (double)n;
                for (int k = 1; k < NMOM; k++) mo[k] = (double)acc[k];
            }
            if (sc.couple) {
                const double M = (double)acc[1];
                if (M > 0.0) {
                    win[0] += (double)acc[2] / M;
                    win[1] += (double)acc[3] / M;
                }
                win[2] += (double)acc[9];
                win[3] += (double)acc[10];
                win[4] += (double)acc[11];
            }
        }
        __syncwarp();
    }

    // ---- back to global memory
    if (act) {
        out.xq[gi] = xq; out.yq[gi] = yq; out.th[gi] = th;
        out.u[gi] = u; out.v[gi] = v; out.w[gi] = w; out.r[gi] = r;
    }
    if (head && sc.couple)
        for (int k = 0; k < NWIN; k++) sc.win[(size_t)k * nc + c] = win[k];
    // an empty cell of the warp: zero moments
    if (lane < pk.y && cj >= 0 && nj == 0) {
        double *mo = sc.mom + (size_t)cj * NMOM;
        for (int k = 0; k < NMOM; k++) mo[k] = 0.0;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep_steps) atomicAdd(&sc.ctrl->deep, (unsigned long long)deep_steps);
}

// ===================================================================== FP64
// Positions are FP64 offsets from the cell origin; minimum image and wrap as
// x - L rint(x / L) and x - L floor(x / L).  Pairs are visited in ascending
// partner index, so each floe sums its contacts in the order the pairs (l < j)
// of the cell are listed.

template <int T>
__global__ void __launch_bounds__(T)
k_cell_step64_brute(DevState64 in, DevState64 out, Phys<double> P, StepCommon sc, int persistent)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int maxn = sc.max_n;
    double *X = reinterpret_cast<double *>(smem);
    double *Y = X + maxn, *U = Y + maxn, *V = U + maxn, *Wv = V + maxn, *Rr = Wv + maxn, *H = Rr + maxn;
    double *red = H + maxn;
    int *sh_item = reinterpret_cast<int *>(red + (T / 32) * NMOM);

    const StepInfo si = step_info(sc);
    double ua, va;
    wind_at(P, si.t, ua, va);
    const double dt = sc.dt;
    const double Lx = sc.g.Lcx, Ly = sc.g.Lcy;
    unsigned deep = 0;
    bool bad = false;

    for (int item = next_item(sc, persistent, sh_item, true); item < sc.ncell;
         item = next_item(sc, persistent, sh_item, false)) {
        const int c = sc.order[item];
        const int o = sc.off[c], n = sc.off[c + 1] - o;
        const int ix = c % sc.g.nx, iy = (c / sc.g.nx) % sc.g.nyr;
        const double X0 = ix * Lx, Y0 = iy * Ly;
        for (int k = threadIdx.x; k < n; k += T) {
            X[k] = in.x[o + k]; Y[k] = in.y[o + k]; U[k] = in.u[o + k]; V[k] = in.v[o + k];
            Wv[k] = in.w[o + k]; Rr[k] = in.r[o + k]; H[k] = in.h[o + k];
        }
        RampCell rc = {1.0, 0.0, 0.0, 0.0};
        if (si.ramp) rc = ramp_cell(sc, c, si.ev);
        __syncthreads();

        double acc[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; k++) acc[k] = 0.0;

        for (int l = threadIdx.x; l < n; l += T) {
            const double xl = X[l], yl = Y[l], ul = U[l], vl = V[l], wl = Wv[l], rl = Rr[l], hl = H[l];
            double fx = 0.0, fy = 0.0, tq = 0.0;
            for (int j = 0; j < n; j++) {
                if (j == l) continue;
                double dx = X[j] - xl, dy = Y[j] - yl;
                dx -= Lx * rint(dx / Lx);
                dy -= Ly * rint(dy / Ly);
                const double d2 = dx * dx + dy * dy;
                contact_add(dx, dy, d2, rl, Rr[j], hl, H[j], U[j] - ul, V[j] - vl, wl, Wv[j], P,
                            fx, fy, tq, deep);
            }
            double uo, vo, zeta;
            ocean_f64(P, X0 + xl, Y0 + yl, uo, vo, zeta);
            double Fdx, Fdy, Td;
            drag_force(P, uo, vo, zeta, ua, va, ul, vl, wl, rl, Fdx, Fdy, Td);
            fx += Fdx; fy += Fdy; tq += Td;
            const double m = P.mass_c * rl * rl * hl;
            const double I = P.inertia_f * m * rl * rl;
            double xn = xl + dt * ul;
            double yn = yl + dt * vl;
            const double th = in.th[o + l] + dt * wl;
            double un = ul + dt * (fx / m);
            double vn = vl + dt * (fy / m);
            double wn = wl + dt * (tq / I);
            xn -= Lx * floor(xn / Lx);
            yn -= Ly * floor(yn / Ly);
            double rn = rl;
            if (si.ramp) {
                rn = rl * rc.g;
                un += rc.du;
                vn += rc.dv;
                wn += rc.dw;
            }
            bad |= !(isfinite(un) && isfinite(vn) && isfinite(wn));
            out.x[o + l] = xn;
            out.y[o + l] = yn;
            out.th[o + l] = th;
            out.u[o + l] = un;
            out.v[o + l] = vn;
            out.w[o + l] = wn;
            if (si.ramp || out.r != in.r) out.r[o + l] = rn;
            add_moments(acc, P.mass_c, P.inertia_f, un, vn, wn, rn, hl, Fdx, Fdy, Td);
        }
        reduce_write<double, T>(acc, red, sc, c, n);
        __syncthreads();
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&sc.ctrl->deep, 1ull);
}

// ============================================================ moments only
// Moments of the current state with zero drag columns (before any step, or
// after the state was replaced).
template <class R, int T>
__global__ void __launch_bounds__(T)
k_cell_moments(const R *u, const R *v, const R *w, const R *r, const R *h, R mass_c, R inertia_f,
               StepCommon sc)
{
    __shared__ double red[(T / 32) * NMOM];
    const int c = blockIdx.x;
    const int o = sc.off[c], n = sc.off[c + 1] - o;
    R acc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; k++) acc[k] = R(0);
    for (int l = threadIdx.x; l < n; l += T)
        add_moments(acc, mass_c, inertia_f, u[o + l], v[o + l], w[o + l], r[o + l], h[o + l], R(0),
                    R(0), R(0));
    StepCommon s2 = sc;
    s2.couple = 0;
    reduce_write<R, T>(acc, red, s2, c, n);
}

}  // namespace

#define MS_T_SWITCH(T, ...)                                       \
    switch (T) {                                                  \
    case 64: { constexpr int TT = 64; __VA_ARGS__; } break;       \
    case 128: { constexpr int TT = 128; __VA_ARGS__; } break;     \
    case 256: { constexpr int TT = 256; __VA_ARGS__; } break;     \
    default: return cudaErrorInvalidValue;                        \
    }

// The shared-memory limit is an attribute of each kernel instance, shared by
// every model in the process: set it once to the device's opt-in maximum
// (a limit, not a reservation) instead of to one launch's need.
// bins per side that a segment can need: nb = sqrt(n) / beta, capped
int seg_nbmax(const CellLaunch &cl, int s)
{
    int nb = (int)(std::sqrt((float)cl.seg_maxn[s]) / cl.bin_beta);
    const int cap = cl.seg_kind[s] == 1 ? 16 : cl.nbmax;
    nb = nb > cap ? cap : nb;
    return nb < 3 ? 3 : nb;
}

static size_t seg_smem(const CellLaunch &cl, int s)
{
    if (cl.seg_kind[s] == 3) return run_block_smem(cl.seg_maxn[s] / RUN_T);
    if (cl.seg_kind[s] == 2) return 4 * pack_region_bytes();
    if (cl.seg_kind[s] == 1 && cl.variant == 3) return 4 * run_region_bytes(cl.seg_maxn[s], seg_nbmax(cl, s));
    if (cl.seg_kind[s] == 1 && cl.variant == 4) return 4 * list_region_bytes(cl.seg_maxn[s], seg_nbmax(cl, s));
    if (cl.seg_kind[s] == 1) return 4 * warp_region_bytes(cl.seg_maxn[s], seg_nbmax(cl, s));
    return smem32_binned(cl.seg_threads[s], cl.seg_maxn[s], seg_nbmax(cl, s));
}

// nsteps fine steps of size class s from step sc.i_local of the interval:
// one launch of a resident kernel (packed cells; warp cells in variant 3),
// else one launch per step
static cudaError_t launch_seg32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                                const StepCommon &sc0, const CellLaunch &cl, int s, cudaStream_t st, int nsteps = 1)
{
    const int items = cl.seg_end[s] - cl.seg_begin[s];
    if (items <= 0) return cudaSuccess;
    const int nbm = seg_nbmax(cl, s);
    const size_t sm = seg_smem(cl, s);
    if (cl.seg_kind[s] == 3) {   // resident blocks (variant 5): one launch for the whole run
        const int K = cl.seg_maxn[s] / RUN_T;
        return launch_run_block(K, in, out, P, sc0, cl.rgroups[s], cl.rngroups[s], cl.ritems,
                                K == 1 ? 0 : (K == 2 ? 1 : 2), nsteps, cl.run_skin, st);
    }
    if (cl.seg_kind[s] == 2) {   // resident in registers: one launch for the whole run
        if (cl.npack <= 0) return cudaSuccess;
        k_cell_run32_packed<4><<<(cl.npack + 3) / 4, 128, sm, st>>>(in, out, P, sc0, cl.pack, cl.npack, nsteps);
        return cudaGetLastError();
    }
    if (cl.seg_kind[s] == 1 && cl.variant == 4 && nsteps == 1) {
        k_cell_step32_wlist<4><<<(items + 3) / 4, 128, sm, st>>>(in, out, P, sc0, cl.bin_beta, cl.seg_begin[s],
                                                                 cl.seg_end[s], cl.seg_maxn[s], nbm, s);
        return cudaGetLastError();
    }
    if (cl.seg_kind[s] == 1 && cl.variant == 3) {
        k_cell_run32_warp<4><<<(items + 3) / 4, 128, sm, st>>>(in, out, P, sc0, nsteps, cl.bin_beta, cl.seg_begin[s],
                                                               cl.seg_end[s], cl.seg_maxn[s], nbm, s);
        return cudaGetLastError();
    }
    if (nsteps > 1) {
        StepCommon sc = sc0;
        for (int i = 0; i < nsteps; i++) {
            sc.i_local = sc0.i_local + i;
            cudaError_t e = launch_seg32(i == 0 ? in : out, out, P, sc, cl, s, st, 1);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const StepCommon &sc = sc0;
    if (cl.seg_kind[s] == 1) {
        k_cell_step32_warp<4><<<(items + 3) / 4, 128, sm, st>>>(in, out, P, sc, cl.bin_beta, cl.seg_begin[s],
                                                                cl.seg_end[s], cl.seg_maxn[s], nbm, s);
        return cudaGetLastError();
    }
    if (cl.variant >= 4) {
        MS_T_SWITCH(cl.seg_threads[s],
                    k_cell_step32_binned<TT, true><<<items, TT, sm, st>>>(in, out, P, sc, cl.bin_beta, cl.seg_begin[s],
                                                                          cl.seg_end[s], cl.seg_maxn[s], nbm, s));
        return cudaGetLastError();
    }
    MS_T_SWITCH(cl.seg_threads[s],
                k_cell_step32_binned<TT><<<items, TT, sm, st>>>(in, out, P, sc, cl.bin_beta, cl.seg_begin[s],
                                                                cl.seg_end[s], cl.seg_maxn[s], nbm, s));
    return cudaGetLastError();
}

size_t cell_step_smem(int precision, const CellLaunch &cl, int max_n, int, int)
{
    const int T = cl.threads;
    if (precision == 0 && cl.variant >= 1) {
        size_t mx = 0;
        for (int s = 0; s < cl.nseg; s++) {
            const size_t sm = seg_smem(cl, s);
            mx = sm > mx ? sm : mx;
        }
        return mx;
    }
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    if (precision == 1) {
        return sizeof(double) * 7 * (size_t)max_n + sizeof(double) * (T / 32) * NMOM + 16;
    }
    return a16(sizeof(float4) * max_n) + a16(sizeof(uint2) * max_n) + a16(sizeof(float) * max_n) +
           sizeof(double) * (T / 32) * NMOM + sizeof(float) * MAXM + 16;
}

cudaError_t cell_step_prepare(int, const CellLaunch &, size_t smem)
{
    static int done = 0;
    static int optin = 0;
    static int limit = 0;
    if (!done) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const void *kern[] = {
            (const void *)k_cell_step32_brute<64>, (const void *)k_cell_step32_brute<128>,
            (const void *)k_cell_step32_brute<256>, (const void *)k_cell_step64_brute<64>,
            (const void *)k_cell_step64_brute<128>, (const void *)k_cell_step64_brute<256>,
            (const void *)k_cell_step32_binned<64>, (const void *)k_cell_step32_binned<128>,
            (const void *)k_cell_step32_binned<256>, (const void *)k_cell_step32_warp<4>,
            (const void *)k_cell_run32_warp<4>, (const void *)k_cell_run32_packed<4>,
            (const void *)k_cell_step32_wlist<4>, (const void *)k_cell_step32_binned<64, true>,
            (const void *)k_cell_step32_binned<128, true>, (const void *)k_cell_step32_binned<256, true>};
        limit = optin;
        if ((e = run_block_prepare()) != cudaSuccess) return e;
        for (const void *k : kern) {
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, k);
            if (e != cudaSuccess) return e;
            const int dyn = optin - (int)fa.sharedSizeBytes;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
            if (e != cudaSuccess) return e;
            limit = dyn < limit ? dyn : limit;
        }
        done = 1;
    }
    return smem <= (size_t)limit ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t cell_fork(const CellLaunch &cl, cudaStream_t st)
{
    cudaError_t e = cudaEventRecord(cl.ev_fork, st);
    for (int s = 0; s < cl.nseg && e == cudaSuccess; s++) e = cudaStreamWaitEvent(cl.side[s], cl.ev_fork, 0);
    return e;
}

cudaError_t cell_join(const CellLaunch &cl, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < cl.nseg && e == cudaSuccess; s++) {
        if ((e = cudaEventRecord(cl.ev_join[s], cl.side[s])) != cudaSuccess) break;
        e = cudaStreamWaitEvent(st, cl.ev_join[s], 0);
    }
    return e;
}

cudaError_t launch_cell_run32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                              const StepCommon &sc, const CellLaunch &cl, int nsteps)
{
    for (int s = 0; s < cl.nseg; s++) {
        cudaError_t e = launch_seg32(in, out, P, sc, cl, s, cl.side[s], nsteps);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cell_step32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                               const StepCommon &sc, const CellLaunch &cl, cudaStream_t st)
{
    if (cl.variant == 1) {
        for (int s = 0; s < cl.nseg; s++) {
            cudaError_t e = launch_seg32(in, out, P, sc, cl, s, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (cl.variant >= 2) {
        // every size class on its own stream: the classes hold disjoint cells,
        // so their kernels overlap and their tails hide each other
        cudaError_t e = cudaEventRecord(cl.ev_fork, st);
        for (int s = 0; s < cl.nseg && e == cudaSuccess; s++) {
            if ((e = cudaStreamWaitEvent(cl.side[s], cl.ev_fork, 0)) != cudaSuccess) break;
            if ((e = launch_seg32(in, out, P, sc, cl, s, cl.side[s])) != cudaSuccess) break;
            if ((e = cudaEventRecord(cl.ev_join[s], cl.side[s])) != cudaSuccess) break;
            e = cudaStreamWaitEvent(st, cl.ev_join[s], 0);
        }
        return e;
    }
    const size_t smem = cell_step_smem(0, cl, sc.max_n, sc.g.nx, sc.g.ny);
    const int grid = cl.persistent ? cl.grid : sc.ncell;
    if (grid <= 0) return cudaSuccess;
    MS_T_SWITCH(cl.threads, k_cell_step32_brute<TT><<<grid, TT, smem, st>>>(in, out, P, sc, cl.persistent));
    return cudaGetLastError();
}

cudaError_t launch_cell_step64(const DevState64 &in, const DevState64 &out, const Phys<double> &P,
                               const StepCommon &sc, const CellLaunch &cl, cudaStream_t st)
{
    const size_t smem = cell_step_smem(1, cl, sc.max_n, sc.g.nx, sc.g.ny);
    const int grid = cl.persistent ? cl.grid : sc.ncell;
    if (grid <= 0) return cudaSuccess;
    MS_T_SWITCH(cl.threads, k_cell_step64_brute<TT><<<grid, TT, smem, st>>>(in, out, P, sc, cl.persistent));
    return cudaGetLastError();
}

cudaError_t launch_cell_moments32(const DevState32 &s, const Phys<float> &P, const StepCommon &sc,
                                  cudaStream_t st)
{
    if (sc.ncell <= 0) return cudaSuccess;
    k_cell_moments<float, 128><<<sc.ncell, 128, 0, st>>>(s.u, s.v, s.w, s.r, s.h, P.mass_c, P.inertia_f, sc);
    return cudaGetLastError();
}

cudaError_t launch_cell_moments64(const DevState64 &s, const Phys<double> &P, const StepCommon &sc,
                                  cudaStream_t st)
{
    if (sc.ncell <= 0) return cudaSuccess;
    k_cell_moments<double, 128><<<sc.ncell, 128, 0, st>>>(s.u, s.v, s.w, s.r, s.h, P.mass_c, P.inertia_f, sc);
    return cudaGetLastError();
}

}  // namespace msd
