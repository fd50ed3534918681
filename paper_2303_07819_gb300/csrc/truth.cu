// truth.cu -- the un-localised DEM over the whole periodic domain (the
// "truth" the paper compares the multiscale model against, Sec. 4), and the
// binning of its floes by coarse cell for the moments.
//
// Every step the floes are re-binned by a GPU counting sort (count -> scan ->
// scatter -> per-bin sort by floe index, so the bin contents and thus the
// force summation order are deterministic).  Floes of radius <= r_split go to
// a grid of bins wider than 2 r_split, larger ones to a grid of bins wider
// than 2 r_max (with a narrow radius distribution r_split = r_max and the
// second grid is empty); a floe visits the bins of the first grid within
// r_l + r_split of its own and the 3 x 3 neighbourhood in the second.  The
// state is double-buffered: the step reads one copy and writes the other.
#include <climits>

#include "common.cuh"
#include "upload.cuh"

namespace msd {

namespace {

constexpr int SCAN_T = 1024;

__global__ void k_scan_blocks(const int *in, int *out, int *bsum, int n)
{
    __shared__ int ws[32];
    const int i = blockIdx.x * SCAN_T + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? ws[warp - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = incl;
}

// exclusive scan of the block sums, in place (nb <= SCAN_T)
__global__ void k_scan_top(int *bsum, int nb)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = threadIdx.x < nb ? bsum[threadIdx.x] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? ws[warp - 1] : 0);
    if (threadIdx.x < nb) bsum[threadIdx.x] = incl - v;
}

__global__ void k_scan_add(int *out, const int *bsum, int n)
{
    const int i = blockIdx.x * SCAN_T + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

__global__ void k_set_int(int *p, int v) { *p = v; }

__global__ void k_scatter(const int *bin, const int *start, int *cursor, int *sorted, long long n)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int b = bin[l];
    sorted[start[b] + atomicAdd(&cursor[b], 1)] = (int)l;
}

// Each bin's floe indices into ascending order, a thread per bin (grids with
// few floes per bin): up to 16 indices sorted in registers, larger bins in
// place in global memory.
__global__ void k_bin_sort_sparse(const int *start, int *sorted, int nbins)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int s = start[b], m = start[b + 1] - s;
    if (m <= 1) return;
    int *bin = sorted + s;
    if (m <= 16) {
        int v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = i < m ? bin[i] : INT_MAX;
        // insertion sort on registers (the unrolled indices keep v in registers)
#pragma unroll
        for (int i = 1; i < 16; i++) {
#pragma unroll
            for (int j = i; j > 0; j--) {
                const int lo = min(v[j - 1], v[j]), hi = max(v[j - 1], v[j]);
                v[j - 1] = lo;
                v[j] = hi;
            }
        }
#pragma unroll
        for (int i = 0; i < 16; i++)
            if (i < m) bin[i] = v[i];
        return;
    }
    for (int i = 1; i < m; i++) {
        const int key = bin[i];
        int j = i - 1;
        while (j >= 0 && bin[j] > key) {
            bin[j + 1] = bin[j];
            j--;
        }
        bin[j + 1] = key;
    }
}

// Each bin's floe indices into ascending order, a warp per bin: every
// index's final place is its rank, the number of smaller indices in the bin
// (indices are distinct), so a lane ranks its entries against the bin's
// entries and all lanes write after all have read.  Bins of up to 32 floes
// rank from registers by shuffles; larger ones read the bin again per entry.
constexpr int SORT_WARPS = 8;

__global__ void __launch_bounds__(SORT_WARPS * 32) k_bin_sort(const int *start, int *sorted, int nbins)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * SORT_WARPS + (threadIdx.x >> 5);
    if (b >= nbins) return;
    const int s = start[b], m = start[b + 1] - s;
    if (m <= 1) return;
    int *bin = sorted + s;
    if (m <= 32) {
        const int key = lane < m ? bin[lane] : INT_MAX;
        int rank = 0;
        for (int i = 0; i < m; i++) rank += __shfl_sync(0xffffffffu, key, i) < key ? 1 : 0;
        __syncwarp();
        if (lane < m) bin[rank] = key;
        return;
    }
    // larger bins: at most 8 entries per lane held in registers until all
    // lanes have ranked theirs (bins above 256 floes fall back to a serial
    // insertion sort by lane 0)
    if (m > 256) {
        if (lane == 0)
            for (int i = 1; i < m; i++) {
                const int key = bin[i];
                int j = i - 1;
                while (j >= 0 && bin[j] > key) {
                    bin[j + 1] = bin[j];
                    j--;
                }
                bin[j + 1] = key;
            }
        return;
    }
    int keys[8], ranks[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
        const int i = lane + 32 * t;
        keys[t] = i < m ? bin[i] : INT_MAX;
        ranks[t] = 0;
    }
    for (int i = 0; i < m; i++) {
        const int other = bin[i];
#pragma unroll
        for (int t = 0; t < 8; t++) ranks[t] += other < keys[t] ? 1 : 0;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 8; t++)
        if (lane + 32 * t < m) bin[ranks[t]] = keys[t];
}

// bin of a fixed-point coordinate: floor(frac * nb) exactly
__device__ __forceinline__ int fbin(uint32_t q, int nb) { return (int)(((unsigned long long)q * (unsigned)nb) >> 32); }

__device__ __forceinline__ int dbin(double x, double L, int nb)
{
    int b = (int)floor(x / (L / nb));
    return b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
}

// bin of floe l: the first grid for radii <= r_split (or r == nullptr), the
// second grid's bins after the first's
__global__ void k_bin32(const uint32_t *xq, const uint32_t *yq, const float *r, TruthBins tb, long long n)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    int b;
    if (!r || r[l] <= tb.r_split) b = fbin(yq[l], tb.nby) * tb.nbx + fbin(xq[l], tb.nbx);
    else b = tb.nbx * tb.nby + fbin(yq[l], tb.nby2) * tb.nbx2 + fbin(xq[l], tb.nbx2);
    tb.bin[l] = b;
    atomicAdd(&tb.count[b], 1);
}

__global__ void k_bin64(const double *x, const double *y, const double *r, double Lx, double Ly, TruthBins tb,
                        long long n)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    int b;
    if (!r || r[l] <= (double)tb.r_split) b = dbin(y[l], Ly, tb.nby) * tb.nbx + dbin(x[l], Lx, tb.nbx);
    else b = tb.nbx * tb.nby + dbin(y[l], Ly, tb.nby2) * tb.nbx2 + dbin(x[l], Lx, tb.nbx2);
    tb.bin[l] = b;
    atomicAdd(&tb.count[b], 1);
}

// ------------------------------------------------------------ truth steps
// Floe l against the rigid walls x = 0 and x = Lx (Sec. 4.4): the contact law
// of Eq. (2.2) with the wall as the partner, a floe at rest without spin, of
// unbounded radius and at least floe l's thickness.  Its edge is the wall
// line, so the overlap is delta = d - r_l (d: the centre's distance to the
// wall, dl and dr below), the lens becomes the segment the line cuts off with
// chord 2 sqrt(r_l^2 - d^2), and the normal n = (-1, 0) or (1, 0) points into
// the wall; the tangent t = (0, n_x).  Adds the force on l.
template <class R>
__device__ __forceinline__ void wall_add(R dl, R dr, R ul, R vl, R wl, R rl, R hl, const Phys<R> &P, R &fx,
                                         R &fy, R &tq, unsigned &deep)
{
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const R d = side == 0 ? dl : dr;
        if (!(d < rl)) continue;
        const R nx = side == 0 ? R(-1) : R(1);
        const R delta = d - rl;
        const R c = d > -rl ? R(2) * sqrt(rl * rl - d * d) : R(2) * rl;
        const R hc = hl * P.inv_h_ref;
        const R vn = -ul * nx;                 // (wall - floe) velocity along n
        R Fn = c * hc * (P.E * delta + P.eta * vn);
        Fn = dmin(Fn, R(0));
        const R vt = -vl * nx - wl * rl;       // along t, minus the floe's rim speed
        R ft = c * hc * P.G * vt;
        const R cap = P.mu * (-Fn);
        ft = dmax(dmin(ft, cap), -cap);
        fx += Fn * nx;
        fy += ft * nx;
        tq += rl * ft;
        deep |= (delta < R(-0.5) * rl) ? 1u : 0u;
    }
}

// The bins along one axis whose floes can touch a floe at coordinate bin b
// reaching `reach` beyond its own bin's edge (k = ceil(reach / bin side)
// bins to either side): offsets o0..o1 from b, or every bin of the axis
// (offsets 0..nb-1 from bin 0, `all`) when that many would wrap onto
// themselves.
struct AxisRange {
    int b0, o0, o1;
    bool all;
};
__device__ __forceinline__ AxisRange axis_range(int b, int nb, float reach_bins)
{
    AxisRange a;
    const int k = (int)ceilf(reach_bins * 1.0001f);   // margin against rounding; bins are wider than 2.0002 r
    if (2 * k + 1 >= nb) {
        a.all = true; a.b0 = 0; a.o0 = 0; a.o1 = nb - 1;
    } else {
        a.all = false; a.b0 = b; a.o0 = -k; a.o1 = k;
    }
    return a;
}

// Visits the bins of one grid (nbx x nby bins from bin index `base`) that
// can hold a partner of a floe at coordinate bins (bx, by) reaching
// (rx, ry) bin sides beyond its own bin, in a fixed order (y, then x), with
// periodic wrap in y and, without walls, in x.
template <class F>
__device__ __forceinline__ void visit_bins(int base, int nbx, int nby, int bx, int by, float rx, float ry, bool walls,
                                           F &&scan_bin)
{
    const AxisRange ax = axis_range(bx, nbx, rx), ay = axis_range(by, nby, ry);
    for (int oy = ay.o0; oy <= ay.o1; oy++) {
        int cy = ay.b0 + oy;
        cy = cy < 0 ? cy + nby : (cy >= nby ? cy - nby : cy);
        for (int ox = ax.o0; ox <= ax.o1; ox++) {
            int cx = ax.b0 + ox;
            if (walls && (cx < 0 || cx >= nbx)) continue;   // no image across a wall
            cx = cx < 0 ? cx + nbx : (cx >= nbx ? cx - nbx : cx);
            scan_bin(base + cy * nbx + cx);
        }
    }
}

__global__ void k_truth32(DevState32 in, DevState32 out, Phys<float> P, TruthArgs a, TruthBins tb)
{
    __shared__ float wind[2];
    if (threadIdx.x == 0) {
        float ua, va;
        wind_at(P, (double)a.step * a.dt, ua, va);
        wind[0] = ua;
        wind[1] = va;
    }
    __syncthreads();
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n) return;
    const float sx = a.k.sx, sy = a.k.sy, isx = a.k.isx, isy = a.k.isy;
    const uint32_t xl = in.xq[l], yl = in.yq[l];
    const float ul = in.u[l], vl = in.v[l], wl = in.w[l], rl = in.r[l], hl = in.h[l];
    const bool walls = a.g.walls != 0;
    float fx = 0.0f, fy = 0.0f, tq = 0.0f;
    unsigned deep = 0;
    auto scan_bin = [&](int cb) {
        for (int k = tb.start[cb]; k < tb.start[cb + 1]; k++) {
            const int j = tb.sorted[k];
            if (j == l) continue;
            // between walls the plain difference (partners up to two bins
            // away may be more than half the domain apart), else the
            // periodic minimum image of the 32-bit fixed point
            const float dx = walls ? (float)((long long)in.xq[j] - (long long)xl) * sx
                                   : (float)(int)(in.xq[j] - xl) * sx;
            const float dy = (float)(int)(in.yq[j] - yl) * sy;
            const float d2 = dx * dx + dy * dy;
            const float rj = in.r[j];
            const float S = rl + rj;
            if (d2 < S * S)
                contact_add(dx, dy, d2, rl, rj, hl, in.h[j], in.u[j] - ul, in.v[j] - vl, wl, in.w[j], P,
                            fx, fy, tq, deep);
        }
    };
    // partners of radius <= r_split in the first grid, within r_l + r_split;
    // larger partners in the second grid (bins wider than 2 r_max: 3 x 3)
    const float Lx = (float)a.g.Lx, Ly = (float)a.g.Ly, reach = rl + tb.r_split;
    visit_bins(0, tb.nbx, tb.nby, fbin(xl, tb.nbx), fbin(yl, tb.nby), reach * tb.nbx / Lx, reach * tb.nby / Ly,
               walls, scan_bin);
    if (tb.nbx2 > 0)
        visit_bins(tb.nbx * tb.nby, tb.nbx2, tb.nby2, fbin(xl, tb.nbx2), fbin(yl, tb.nby2), 0.99f, 0.99f, walls,
                   scan_bin);   // bins wider than 2 r_max: every partner within one bin
    // ocean at the domain fraction, phases in cycles per domain
    const float xf = (float)xl * 2.3283064365386963e-10f, yf = (float)yl * 2.3283064365386963e-10f;
    float uo = P.uo_x, vo = P.uo_y, zeta = 0.0f;
    for (int m = 0; m < P.n_modes; m++) {
        float cyc = P.kdx[m] * xf + P.kdy[m] * yf + P.mCyc[m];
        cyc -= floorf(cyc);
        float s, c;
        sincospif(2.0f * cyc, &s, &c);
        uo -= P.mAu[m] * c;
        vo += P.mAv[m] * c;
        zeta -= P.mAz[m] * s;
    }
    if (walls) {
        // distances to the walls from the fixed point: exact integers, one rounding
        const float dl = (float)xl * sx, dr = (float)(4294967296ll - (long long)xl) * sx;
        wall_add(dl, dr, ul, vl, wl, rl, hl, P, fx, fy, tq, deep);
    }
    float Fdx, Fdy, Td;
    drag_force(P, uo, vo, zeta, wind[0], wind[1], ul, vl, wl, rl, Fdx, Fdy, Td);
    fx += Fdx; fy += Fdy; tq += Td;
    const float dt = a.k.dt;
    const float m = P.mass_c * rl * rl * hl;
    const float I = P.inertia_f * m * rl * rl;
    if (walls) {
        // reading: a centre that would pass a wall stays on it (in a stable run
        // the wall's contact force stops the floe long before)
        long long xn = (long long)xl + __float2int_rn(dt * ul * isx);
        xn = xn < 0 ? 0 : (xn > 4294967295ll ? 4294967295ll : xn);
        out.xq[l] = (uint32_t)xn;
    } else {
        out.xq[l] = xl + (uint32_t)__float2int_rn(dt * ul * isx);
    }
    out.yq[l] = yl + (uint32_t)__float2int_rn(dt * vl * isy);
    out.th[l] = in.th[l] + dt * wl;
    const float un = ul + dt * (fx / m), vn = vl + dt * (fy / m), wn = wl + dt * (tq / I);
    out.u[l] = un;
    out.v[l] = vn;
    out.w[l] = wn;
    out.r[l] = rl;
    out.h[l] = hl;
    float *fd = reinterpret_cast<float *>(a.fd);
    fd[l] = Fdx; fd[a.n + l] = Fdy; fd[2 * a.n + l] = Td;
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn))) atomicOr(&a.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&a.ctrl->deep, 1ull);
}

__global__ void k_truth64(DevState64 in, DevState64 out, Phys<double> P, TruthArgs a, TruthBins tb)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n) return;
    const double Lx = a.g.Lx, Ly = a.g.Ly;
    const double xl = in.x[l], yl = in.y[l], ul = in.u[l], vl = in.v[l], wl = in.w[l], rl = in.r[l],
                 hl = in.h[l];
    const bool walls = a.g.walls != 0;
    double fx = 0.0, fy = 0.0, tq = 0.0;
    unsigned deep = 0;
    auto scan_bin = [&](int cb) {
        for (int k = tb.start[cb]; k < tb.start[cb + 1]; k++) {
            const int j = tb.sorted[k];
            if (j == l) continue;
            double dx = in.x[j] - xl, dy = in.y[j] - yl;
            if (!walls) dx -= Lx * rint(dx / Lx);
            dy -= Ly * rint(dy / Ly);
            const double d2 = dx * dx + dy * dy;
            contact_add(dx, dy, d2, rl, in.r[j], hl, in.h[j], in.u[j] - ul, in.v[j] - vl, wl, in.w[j], P,
                        fx, fy, tq, deep);
        }
    };
    const double reach = rl + (double)tb.r_split;
    visit_bins(0, tb.nbx, tb.nby, dbin(xl, Lx, tb.nbx), dbin(yl, Ly, tb.nby), (float)(reach * tb.nbx / Lx),
               (float)(reach * tb.nby / Ly), walls, scan_bin);
    if (tb.nbx2 > 0)
        visit_bins(tb.nbx * tb.nby, tb.nbx2, tb.nby2, dbin(xl, Lx, tb.nbx2), dbin(yl, Ly, tb.nby2), 0.99f, 0.99f,
                   walls, scan_bin);   // bins wider than 2 r_max: every partner within one bin
    double uo, vo, zeta;
    ocean_f64(P, xl, yl, uo, vo, zeta);
    double ua, va;
    wind_at(P, (double)a.step * a.dt, ua, va);
    if (walls) wall_add(xl, Lx - xl, ul, vl, wl, rl, hl, P, fx, fy, tq, deep);
    double Fdx, Fdy, Td;
    drag_force(P, uo, vo, zeta, ua, va, ul, vl, wl, rl, Fdx, Fdy, Td);
    fx += Fdx; fy += Fdy; tq += Td;
    const double dt = a.dt;
    const double m = P.mass_c * rl * rl * hl;
    const double I = P.inertia_f * m * rl * rl;
    double xn = xl + dt * ul, yn = yl + dt * vl;
    if (!walls) xn -= Lx * floor(xn / Lx);
    else xn = fmin(fmax(xn, 0.0), Lx);   // reading: a centre that would pass a wall stays on it
    yn -= Ly * floor(yn / Ly);
    out.x[l] = xn;
    out.y[l] = yn;
    out.th[l] = in.th[l] + dt * wl;
    const double un = ul + dt * (fx / m), vn = vl + dt * (fy / m), wn = wl + dt * (tq / I);
    out.u[l] = un;
    out.v[l] = vn;
    out.w[l] = wn;
    out.r[l] = rl;
    out.h[l] = hl;
    double *fd = reinterpret_cast<double *>(a.fd);
    fd[l] = Fdx; fd[a.n + l] = Fdy; fd[2 * a.n + l] = Td;
    if (!(isfinite(un) && isfinite(vn) && isfinite(wn))) atomicOr(&a.ctrl->err, ERR_NONFINITE);
    if (deep) atomicAdd(&a.ctrl->deep, 1ull);
}

// --------------------------------------------------------- truth moments
// One thread per coarse cell sums its floes in ascending floe index, in FP64.
template <class R>
__global__ void k_truth_cell_moments(const R *u, const R *v, const R *w, const R *r, const R *h, const R *fd,
                                     long long n, double mass_c, double inertia_f, const int *start,
                                     const int *sorted, int ncell, double *mom)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double mo[NMOM];
    for (int k = 0; k < NMOM; k++) mo[k] = 0.0;
    for (int k = start[c]; k < start[c + 1]; k++) {
        const int l = sorted[k];
        const double rl = r[l], hl = h[l], ul = u[l], vl = v[l], wl = w[l];
        const double m = mass_c * rl * rl * hl;
        const double I = inertia_f * m * rl * rl;
        mo[0] += 1.0;
        mo[1] += m;
        mo[2] += m * ul;
        mo[3] += m * vl;
        mo[4] += I;
        mo[5] += I * wl;
        mo[6] += 3.14159265358979323846 * rl * rl;
        mo[7] += m * ul * ul;
        mo[8] += m * vl * vl;
        mo[9] += fd[l];
        mo[10] += fd[n + l];
        mo[11] += fd[2 * n + l];
    }
    for (int k = 0; k < NMOM; k++) mom[(size_t)c * NMOM + k] = mo[k];
}

template <class BinF>
cudaError_t counting_sort(TruthBins &b, long long n, BinF binf, cudaStream_t st)
{
    const int nbins = b.nbins();
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.count, 0, sizeof(int) * nbins, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.cursor, 0, sizeof(int) * nbins, st)) != cudaSuccess) return e;
    if (n > 0) binf();
    if ((e = bins_scan(b, nbins, st)) != cudaSuccess) return e;
    const int T = 256;
    if (n > 0) k_scatter<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.bin, b.start, b.cursor, b.sorted, n);
    if (n < 4LL * nbins)   // few floes per bin on average: a thread per bin
        k_bin_sort_sparse<<<(nbins + T - 1) / T, T, 0, st>>>(b.start, b.sorted, nbins);
    else
        k_bin_sort<<<(nbins + SORT_WARPS - 1) / SORT_WARPS, SORT_WARPS * 32, 0, st>>>(b.start, b.sorted, nbins);
    return cudaGetLastError();
}

}  // namespace

// ---- the floes of a model grouped by cell (ms_init)

// exclusive scan of n ints (in place allowed): per-block scans, the block
// totals scanned the same way, then added back
static cudaError_t scan_exclusive(const int *in, int *out, long long n, int *tmp, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + SCAN_T - 1) / SCAN_T;
    k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, tmp, (int)n);
    if (nb > 1) {
        const cudaError_t e = scan_exclusive(tmp, tmp, nb, tmp + nb, st);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)nb, SCAN_T, 0, st>>>(out, tmp, (int)n);
    }
    return cudaGetLastError();
}

long long sort_scan_ints(long long n)
{
    long long total = 1;
    while (n > 1) {
        n = (n + SCAN_T - 1) / SCAN_T;
        total += n;
    }
    return total + 1;
}

namespace {

constexpr int RANK_T = 256;
constexpr int RANK_MAX = 4096;   // the largest cell a model takes

// A block per cell: the cell's caller indices into ascending order, each
// entry placed at its rank (the number of smaller indices; they are
// distinct).  Cells above RANK_MAX floes are left as scattered (ms_init
// rejects them before this runs).
__global__ void __launch_bounds__(RANK_T) k_cell_rank_sort(const int *off, int *orig, int ncell)
{
    __shared__ int keys[RANK_MAX];
    const int c = blockIdx.x;
    if (c >= ncell) return;
    const int s = off[c], m = off[c + 1] - s;
    if (m <= 1 || m > RANK_MAX) return;
    for (int i = threadIdx.x; i < m; i += RANK_T) keys[i] = orig[s + i];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += RANK_T) {
        const int key = keys[i];
        int rank = 0;
        for (int j = 0; j < m; j++) rank += keys[j] < key ? 1 : 0;
        orig[s + rank] = key;
    }
}

}  // namespace

cudaError_t sort_by_cell(const int *cell_of, const int *count, int *off, int *cursor, int *orig, int *tmp,
                         int ncell, long long n, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st);
    if (e == cudaSuccess) e = scan_exclusive(count, off, ncell, tmp, st);
    if (e != cudaSuccess) return e;
    k_set_int<<<1, 1, 0, st>>>(off + ncell, (int)n);
    const int T = 256;
    if (n > 0) k_scatter<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(cell_of, off, cursor, orig, n);
    if (n > 0 && ncell > 0) k_cell_rank_sort<<<ncell, RANK_T, 0, st>>>(off, orig, ncell);
    return cudaGetLastError();
}

cudaError_t bins_scan(TruthBins &b, int nbins, cudaStream_t st)
{
    const int nb = (nbins + SCAN_T - 1) / SCAN_T;
    if (nb > SCAN_T) return cudaErrorInvalidValue;
    k_scan_blocks<<<nb, SCAN_T, 0, st>>>(b.count, b.start, b.scan_tmp, nbins);
    k_scan_top<<<1, SCAN_T, 0, st>>>(b.scan_tmp, nb);
    k_scan_add<<<nb, SCAN_T, 0, st>>>(b.start, b.scan_tmp, nbins);
    return cudaGetLastError();
}

int truth_launches(const TruthBins &) { return 2 /*memsets*/ + 1 + 3 + 1 + 1 + 1; }

cudaError_t launch_truth_step32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                                const TruthArgs &a, TruthBins &b, cudaStream_t st)
{
    const int T = 128;
    const unsigned G = (unsigned)((a.n + T - 1) / T);
    cudaError_t e = counting_sort(b, a.n, [&] {
        k_bin32<<<G, T, 0, st>>>(in.xq, in.yq, in.r, b, a.n);
    }, st);
    if (e != cudaSuccess) return e;
    if (a.n > 0) k_truth32<<<G, T, 0, st>>>(in, out, P, a, b);
    return cudaGetLastError();
}

cudaError_t launch_truth_step64(const DevState64 &in, const DevState64 &out, const Phys<double> &P,
                                const TruthArgs &a, TruthBins &b, cudaStream_t st)
{
    const int T = 256;
    const unsigned G = (unsigned)((a.n + T - 1) / T);
    cudaError_t e = counting_sort(b, a.n, [&] {
        k_bin64<<<G, T, 0, st>>>(in.x, in.y, in.r, a.g.Lx, a.g.Ly, b, a.n);
    }, st);
    if (e != cudaSuccess) return e;
    if (a.n > 0) k_truth64<<<G, T, 0, st>>>(in, out, P, a, b);
    return cudaGetLastError();
}

cudaError_t launch_truth_moments32(const DevState32 &s, const Phys<float> &P, const TruthArgs &a,
                                   TruthBins &cells, double *mom, cudaStream_t st)
{
    const int T = 256;
    const unsigned G = (unsigned)((a.n + T - 1) / T);
    cudaError_t e = counting_sort(cells, a.n, [&] {
        k_bin32<<<G, T, 0, st>>>(s.xq, s.yq, nullptr, cells, a.n);
    }, st);
    if (e != cudaSuccess) return e;
    const int nc = cells.nbx * cells.nby;
    k_truth_cell_moments<float><<<(nc + 127) / 128, 128, 0, st>>>(
        s.u, s.v, s.w, s.r, s.h, reinterpret_cast<const float *>(a.fd), a.n, (double)P.mass_c,
        (double)P.inertia_f, cells.start, cells.sorted, nc, mom);
    return cudaGetLastError();
}

cudaError_t launch_truth_moments64(const DevState64 &s, const Phys<double> &P, const TruthArgs &a,
                                   TruthBins &cells, double *mom, cudaStream_t st)
{
    const int T = 256;
    const unsigned G = (unsigned)((a.n + T - 1) / T);
    cudaError_t e = counting_sort(cells, a.n, [&] {
        k_bin64<<<G, T, 0, st>>>(s.x, s.y, nullptr, a.g.Lx, a.g.Ly, cells, a.n);
    }, st);
    if (e != cudaSuccess) return e;
    const int nc = cells.nbx * cells.nby;
    k_truth_cell_moments<double><<<(nc + 127) / 128, 128, 0, st>>>(
        s.u, s.v, s.w, s.r, s.h, reinterpret_cast<const double *>(a.fd), a.n, P.mass_c, P.inertia_f,
        cells.start, cells.sorted, nc, mom);
    return cudaGetLastError();
}

// ----------------------------------------------- moments without allocating
// A variant of the per-cell moment binning above whose working memory (the
// counting sort's counts, starts, cursors and the sorted floe list) lives in
// one file-scope device array instead of buffers from cudaMalloc, for callers
// that must not allocate device memory while they run (see msdem.h).  Every
// call on a device reuses the same array: the counts and cursors are cleared
// at the start of each call, and two calls that run on the GPU at the same
// time corrupt each other.

namespace {

// cell of a caller's floe: each coordinate wrapped into [0, L) by
// X - L floor(X / L), then the half-open cell floor(X / (L / n)), clamped
// (rounding can put a wrapped X on L itself) -- the assignment ms_init makes
__device__ __forceinline__ int wrap_cell(double X, double L, int n)
{
    const double Xw = X - L * floor(X / L);
    int i = (int)floor(Xw / (L / n));
    return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

__global__ void k_bin_wrap64(const double *x, const double *y, double Lx, double Ly, TruthBins tb, long long n)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int b = wrap_cell(y[l], Ly, tb.nby) * tb.nbx + wrap_cell(x[l], Lx, tb.nbx);
    tb.bin[l] = b;
    atomicAdd(&tb.count[b], 1);
}

}  // namespace

}  // namespace msd

// Scratch of ms_cell_moments_noalloc: 3 * NA_CELLS + 1 + NA_SCAN ints for the
// cell counts, starts and cursors plus the scan's block sums, then 2 * NA_FLOES
// ints for each floe's cell and the floes sorted by cell (about 2.2 MB).
#define MS_NA_FLOES (1 << 18)
#define MS_NA_CELLS (1 << 14)
#define MS_NA_SCAN ((MS_NA_CELLS + 1 + 1023) / 1024)
static __device__ __align__(256) int ms_noalloc_scratch[3 * MS_NA_CELLS + 1 + MS_NA_SCAN + 2 * MS_NA_FLOES];

namespace msd {

long long noalloc_max_floes() { return MS_NA_FLOES; }
int noalloc_max_cells() { return MS_NA_CELLS; }

// Device address of the scratch array on the current device.  The address a
// host program sees for the symbol is only a host-side placeholder; the device
// address is looked up on every call, with the caller's device current, so a
// context that was torn down and created again (where the module may load at
// another address) never gets a stale pointer.
static cudaError_t noalloc_scratch(int **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, ms_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = reinterpret_cast<int *>(p);
    return cudaSuccess;
}

cudaError_t noalloc_cell_moments(const Geom &g, double mass_c, double inertia_f, long long n, const double *x,
                                 const double *y, const double *u, const double *v, const double *w,
                                 const double *r, const double *h, const double *fd, double *mom,
                                 cudaStream_t st)
{
    int *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return e;
    TruthBins b{};
    b.nbx = g.nx;
    b.nby = g.ny;
    const int nbins = g.nx * g.ny;
    b.count = base;
    b.start = b.count + MS_NA_CELLS;
    b.cursor = b.start + MS_NA_CELLS + 1;
    b.scan_tmp = b.cursor + MS_NA_CELLS;
    b.bin = b.scan_tmp + MS_NA_SCAN;
    b.sorted = b.bin + MS_NA_FLOES;
    b.nscan_blocks = (nbins + 1023) / 1024;
    k_set_int<<<1, 1, 0, st>>>(b.start + nbins, (int)n);
    const int T = 256;
    const unsigned G = (unsigned)((n + T - 1) / T);
    e = counting_sort(b, n, [&] {
        k_bin_wrap64<<<G, T, 0, st>>>(x, y, g.Lx, g.Ly, b, n);
    }, st);
    if (e != cudaSuccess) return e;
    k_truth_cell_moments<double><<<(nbins + 127) / 128, 128, 0, st>>>(u, v, w, r, h, fd, n, mass_c, inertia_f,
                                                                     b.start, b.sorted, nbins, mom);
    return cudaGetLastError();
}

}  // namespace msd
