// hybrid.cu -- closure-plus-fallback coarse intervals, and the training data
// for the closure.
//
// Not in the paper: a learned model of each cell's bulk feedback (the drag
// tendencies that the coarse moment equations, Eq. 2.26, take from the cell's
// DEM, Sec. 3.2) lets a cell skip its DEM for a coarse interval.  At the start
// of every interval each cell's features go through the network; a residual
// check compares the prediction with the mean-field drag of the cell-mean
// velocity and tests the features against the range seen in training; cells
// that fail run the particle step (the fallback), the others take their
// pending coarse increments at once and report the predicted tendencies to
// the coarse step.  The particle path judges the network: after every DEM
// interval of a cell the network's prediction for that interval is compared
// with the cell's measured drag, and only a cell whose last check passed, and
// that has run at most CLOSURE_MAX_RUN closure intervals since, may take the
// closure.  The features include the cell's drag at the interval's start
// (the drag moment columns of the step that ended the interval before, or
// the prediction if it ran the closure): a cell's drag depends on how its
// floes' velocities and spins spread about the means, which the other
// moments do not carry but which changes slowly over an interval.
#include "common.cuh"
#include "fixsum.cuh"

namespace msd {

namespace {

constexpr int NF = NFEAT;   // features per cell
constexpr int NT = 4;    // targets per cell

// Mean share of a coarse increment that the gradual updates have applied,
// averaged over the N0 steps of an interval: updates after steps n_t, 2 n_t,
// ..., N0 each add n_t / N0, so after step k the share is floor(k / n_t) n_t / N0.
__host__ __device__ inline double ramp_mean_share(int N0, int n_t)
{
    double s = 0.0;
    for (int k = 1; k <= N0; k++) s += (double)(k / n_t) * n_t / N0;
    return s / N0;
}

// [rho, ubar, vbar, wbar, var u, var v, u_o, v_o, div u_o, curl u_o, u_a, v_a,
//  the cell's drag per unit mass (x, y) and drag torque per unit inertia at
//  the interval's start (moment columns 9-11 of the step that ended the
//  interval before; a closure cell's are its predicted ones), and the rate
//  of change of the velocity variance over the interval before] (ocean at
// the cell centre, wind at the start of the interval; the last four are zero
// when the interval before computed no tendencies).  The mean velocity and
// spin are the interval means the gradual updates produce: the cell's
// current means plus the mean share of its pending increments.
// The steady forcing at each cell centre: ocean u, v, divergence and curl
// (the ocean does not change in time), computed once per attachment.
__global__ void k_ocean_at_centres(int ncell, Geom g, Phys<double> P, double *oc)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int ix = c % g.nx, iy = (c / g.nx) % g.nyr;
    double uo, vo, zeta;
    ocean_f64(P, (ix + 0.5) * g.Lcx, (iy + 0.5) * g.Lcy, uo, vo, zeta);
    oc[(size_t)c * 4] = uo;
    oc[(size_t)c * 4 + 1] = vo;
    oc[(size_t)c * 4 + 2] = ocean_div_f64(P, (ix + 0.5) * g.Lcx, (iy + 0.5) * g.Lcy);
    oc[(size_t)c * 4 + 3] = zeta;
}

__global__ void k_features(const double *mom, const double *tgt, int ncell, Geom g, Phys<double> P,
                           const Ctrl *ctrl, double dt, double share, const float *Ylag, const double *oc, float *X)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double *mo = mom + (size_t)c * NMOM;
    const double Ac = g.Lcx * g.Lcy;
    const double M = mo[1], I = mo[4];
    const double ub0 = M > 0.0 ? mo[2] / M : 0.0, vb0 = M > 0.0 ? mo[3] / M : 0.0;
    const double wb0 = I > 0.0 ? mo[5] / I : 0.0;
    const double su = M > 0.0 ? fmax(mo[7] / M - ub0 * ub0, 0.0) : 0.0;
    const double sv = M > 0.0 ? fmax(mo[8] / M - vb0 * vb0, 0.0) : 0.0;
    const double sh = ctrl->have_tgt ? share : 0.0;
    const double ub = ub0 + sh * tgt[ncell + c], vb = vb0 + sh * tgt[2 * ncell + c], wb = wb0 + sh * tgt[3 * ncell + c];
    const double uo = oc[(size_t)c * 4], vo = oc[(size_t)c * 4 + 1], div = oc[(size_t)c * 4 + 2],
                 zeta = oc[(size_t)c * 4 + 3];
    double ua, va;
    wind_at(P, (double)ctrl->base * dt, ua, va);
    const bool lag = ctrl->lag_mark == ctrl->base + 1;
    const double f[12] = {M / Ac, ub, vb, wb, su, sv, uo, vo, div, zeta, ua, va};
    for (int k = 0; k < 12; k++) X[(size_t)c * NF + k] = (float)f[k];
    const double d[3] = {M > 0.0 ? mo[9] / M : 0.0, M > 0.0 ? mo[10] / M : 0.0, I > 0.0 ? mo[11] / I : 0.0};
    for (int k = 0; k < 3; k++) X[(size_t)c * NF + 12 + k] = lag ? (float)d[k] : 0.0f;
    X[(size_t)c * NF + 15] = lag ? Ylag[(size_t)c * NT + 3] : 0.0f;
}

// Targets of the interval just run: window means of the cell's total drag per
// unit mass (x, y), of its drag torque per unit inertia, and the rate of change
// of the velocity variance over the interval.  A closure cell's are its
// predicted ones (is_closure, Yuse; nullptr: every cell ran its DEM).  They
// are kept as the next interval's lagged features (Ylag, marked valid for
// the interval that starts at base + N0) and, if Y is given, returned.
// With the network's prediction for the interval (Yp, nerr, age non-null),
// a DEM cell also records the network's relative drag error on it (nerr,
// floor: floor_acc) and resets its closure run (age); a closure cell extends
// its run.
__global__ void k_collect_targets(const double *mom0, const double *mom1, const double *win, int ncell, int N0,
                                  double dT, const int *is_closure, const float *Yuse, Ctrl *ctrl, float *Ylag,
                                  float *Y, const float *Yp, double floor_acc, float *nerr, int *age)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) ctrl->lag_mark = ctrl->base + N0 + 1;
    if (c >= ncell) return;
    if (is_closure && is_closure[c]) {
        for (int k = 0; k < NT; k++) {
            Ylag[(size_t)c * NT + k] = Yuse[(size_t)c * NT + k];
            if (Y) Y[(size_t)c * NT + k] = Yuse[(size_t)c * NT + k];
        }
        if (age) age[c] += 1;
        return;
    }
    const double *a = mom0 + (size_t)c * NMOM, *b = mom1 + (size_t)c * NMOM;
    const double M0 = a[1], I0 = a[4];
    auto var = [](const double *m) {
        if (!(m[1] > 0.0)) return 0.0;
        const double u = m[2] / m[1], v = m[3] / m[1];
        return fmax(m[7] / m[1] - u * u, 0.0) + fmax(m[8] / m[1] - v * v, 0.0);
    };
    const float y[NT] = {M0 > 0.0 ? (float)(win[2 * ncell + c] / N0 / M0) : 0.0f,
                         M0 > 0.0 ? (float)(win[3 * ncell + c] / N0 / M0) : 0.0f,
                         I0 > 0.0 ? (float)(win[4 * ncell + c] / N0 / I0) : 0.0f,
                         (float)((var(b) - var(a)) / dT)};
    for (int k = 0; k < NT; k++) {
        Ylag[(size_t)c * NT + k] = y[k];
        if (Y) Y[(size_t)c * NT + k] = y[k];
    }
    if (Yp && nerr && age) {
        const double ex = (double)Yp[(size_t)c * NT] - y[0], ey = (double)Yp[(size_t)c * NT + 1] - y[1];
        const double ym = sqrt((double)y[0] * y[0] + (double)y[1] * y[1]);
        nerr[c] = M0 > 0.0 ? (float)(sqrt(ex * ex + ey * ey) / (ym + floor_acc)) : 0.0f;
        age[c] = 0;
    }
}

// Mean-field tendencies of a cell: the drag of Eq. 2.1c-d evaluated at the
// cell-mean velocity and spin, per unit mass and inertia (mean thickness
// M / (rho_ice sum pi r^2)); no change of the variance.
__device__ __forceinline__ void meanfield(const float *x, const double *mo, const Phys<double> &P, double rho_ice,
                                          double *y)
{
    const double area = mo[6];
    const double hbar = (area > 0.0 && mo[1] > 0.0) ? mo[1] / (rho_ice * area) : 1.0;
    const double ko = P.drag_o / (3.14159265358979323846 * rho_ice * hbar);
    const double ka = P.drag_a / (3.14159265358979323846 * rho_ice * hbar);
    const double dou = x[6] - x[1], dov = x[7] - x[2];
    const double dau = x[10] - x[1], dav = x[11] - x[2];
    const double so = sqrt(dou * dou + dov * dov), sa = sqrt(dau * dau + dav * dav);
    const double dw = 0.5 * x[9] - x[3];
    y[0] = ko * dou * so + ka * dau * sa;
    y[1] = ko * dov * so + ka * dav * sa;
    y[2] = ko * dw * fabs(dw) / P.inertia_f;
    y[3] = 0.0;
}

// closure or particle for each cell; the tendencies the coarse step will see
__global__ void k_classify(const float *X, float *Yp, const double *mom, int ncell, Phys<double> P,
                           double rho_ice, const float *box, double tol, int mode, const Ctrl *ctrl,
                           const float *nerr, const int *age, int *is_closure, float *Yuse,
                           unsigned long long *closure_count)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const float *x = X + (size_t)c * NF;
    const double *mo = mom + (size_t)c * NMOM;
    double mf[4];
    meanfield(x, mo, P, rho_ice, mf);
    if (mode == 2) {
        // the network gives the change from features 12-15 (the drag at the
        // interval's start, the variance rate of the interval before); from
        // here on Yp holds the tendencies themselves (without an interval
        // before there is nothing to add to, and nothing to check)
        float *yp = Yp + (size_t)c * NT;
        const bool lag = ctrl->lag_mark == ctrl->base + 1;
        for (int k = 0; k < NT; k++) yp[k] = lag ? yp[k] + x[12 + k] : 3.0e38f;
    }
    int closure = 0;
    float y[NT] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (ctrl->have_tgt) {
        if (!(mo[1] > 0.0)) {
            closure = 1;      // an empty cell has nothing to step
        } else if (mode == 1) {
            closure = 1;
            for (int k = 0; k < NT; k++) y[k] = (float)mf[k];
        } else if (ctrl->lag_mark == ctrl->base + 1) {   // the network needs last interval's tendencies
            bool inside = true;
            for (int k = 0; k < NF; k++)
                inside &= (x[k] >= box[k]) && (x[k] <= box[NF + k]);
            const float *yp = Yp + (size_t)c * NT;
            // the residual check: the network's drag error on this cell's last
            // DEM interval, and a bounded run of closure intervals since
            closure = inside && nerr[c] <= tol && age[c] < CLOSURE_MAX_RUN;
            for (int k = 0; k < NT; k++) y[k] = yp[k];
        }
    }
    is_closure[c] = closure;
    for (int k = 0; k < NT; k++) Yuse[(size_t)c * NT + k] = y[k];
    const unsigned bal = __ballot_sync(__activemask(), closure != 0);
    if ((threadIdx.x & 31) == __ffs(__activemask()) - 1 && bal) atomicAdd(closure_count, (unsigned long long)__popc(bal));
}

// Per size class (one block each), the particle cells of the class, in their
// processing order, packed at the front of the class's range.
__global__ void k_compact(const int *order, const int *seg_begin, const int *seg_end, const int *is_closure,
                          int *order2, int *live, unsigned seg_mask)
{
    __shared__ int ws[33];
    const int s = blockIdx.x;
    if (!((seg_mask >> s) & 1u)) return;       // a class whose kernels skip closure cells themselves
    const int b = seg_begin[s], e = seg_end[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = 0, nclos = 0;
    for (int i0 = b; i0 < e; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int c = i < e ? order[i] : -1;
        const int part = (c >= 0 && !is_closure[c]) ? 1 : 0;
        nclos += (c >= 0 && !part) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, part);
        if (lane == 0) ws[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                const int t = ws[w];
                ws[w] = acc;
                acc += t;
            }
            ws[32] = acc;
        }
        __syncthreads();
        if (part) order2[b + base + ws[warp] + __popc(bal & ((1u << lane) - 1u))] = c;
        base += ws[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) live[s] = base;
}

// Cells that share a block run it for the interval's whole length, so a
// closure cell saves time only when the cells beside it take the closure
// too: a group keeps its closure cells only if every cell of it that holds
// floes takes the closure.  A thread per group.
__global__ void k_group_veto(const int4 *groups, int ngroups, const int4 *items, const int *off, int *is_closure,
                             unsigned long long *closure_count)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const int4 gd = groups[g];
    bool all = true;
    for (int i = 0; i < gd.y; i++) {
        const int c = items[gd.x + i].x;
        all &= off[c + 1] == off[c] || is_closure[c] != 0;
    }
    if (all) return;
    unsigned long long dropped = 0;
    for (int i = 0; i < gd.y; i++) {
        const int c = items[gd.x + i].x;
        if (off[c + 1] > off[c] && is_closure[c]) {
            is_closure[c] = 0;
            dropped++;
        }
    }
    if (dropped) atomicAdd(closure_count, 0ull - dropped);
}

// A closure cell runs the interval without its DEM.  It reports to the coarse
// step what the particle path would: window-mean velocity = current mean +
// mean share of the pending increment + the predicted drag acting for the mean
// elapsed time (N0 + 1)/(2 N0) dT, and the predicted drag as the window's drag
// sums.  Its floes end the interval where the particle path would take them:
// the full increments plus dT times the predicted tendencies (uniform shifts),
// the velocity spread scaled to the predicted variance, the radius scale
// (bounded to [0.5, 2] for one interval) applied.  A warp per cell; its
// moments are the exact fixed-point sums of the FP32 values the resident
// cell kernels sum for a DEM cell (fixsum.cuh).
constexpr int CA_WARPS = 4;

__global__ void __launch_bounds__(32 * CA_WARPS)
k_closure_apply(DevState32 st, Phys<float> P, const int *off, const int *is_closure, const float *Yuse,
                double *mom, double *win, double *tgt, int ncell, int N0, double dT, double share)
{
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * CA_WARPS + (threadIdx.x >> 5);
    if (c >= ncell || !is_closure[c]) return;
    const int o = off[c], n = off[c + 1] - o;
    double *mo = mom + (size_t)c * NMOM;
    const double M = mo[1];
    const double ub = M > 0.0 ? mo[2] / M : 0.0, vb = M > 0.0 ? mo[3] / M : 0.0;
    const double var = M > 0.0 ? fmax(mo[7] / M - ub * ub, 0.0) + fmax(mo[8] / M - vb * vb, 0.0) : 0.0;
    const float *y = Yuse + (size_t)c * 4;
    const double nv = var + dT * (double)y[3];
    const float fs = var > 0.0 ? (float)sqrt(fmax(nv, 0.0) / var) : 1.0f;
    const double sc = fmin(fmax(tgt[c], 0.5), 2.0);
    const double dux = tgt[ncell + c], duy = tgt[2 * ncell + c], dw = tgt[3 * ncell + c];
    const float s = (float)sc;
    const float du = (float)(dux + dT * y[0]), dv = (float)(duy + dT * y[1]), dww = (float)(dw + dT * y[2]);
    const float ubf = (float)ub, vbf = (float)vb;
    for (int l = lane; l < n; l += 32) {
        const int i = o + l;
        st.r[i] *= s;
        st.u[i] = ubf + du + fs * (st.u[i] - ubf);
        st.v[i] = vbf + dv + fs * (st.v[i] - vbf);
        st.w[i] += dww;
    }
    // moment columns 1-8 of the new state (each lane reads the floes it wrote)
    auto val = [&](int i, int q) -> float {
        const float r = st.r[i], h = st.h[i], m = P.mass_c * r * r * h, I = P.inertia_f * m * r * r;
        switch (q) {
        case 0: return m;
        case 1: return m * st.u[i];
        case 2: return m * st.v[i];
        case 3: return I;
        case 4: return I * st.w[i];
        case 5: return 3.14159265358979323846f * r * r;
        case 6: return m * st.u[i] * st.u[i];
        default: return m * st.v[i] * st.v[i];
        }
    };
    int e[8];
#pragma unroll
    for (int q = 0; q < 8; q++) e[q] = FIX_NONE;
    for (int l = lane; l < n; l += 32)
#pragma unroll
        for (int q = 0; q < 8; q++) e[q] = max(e[q], fix_exp(fix_counted(val(o + l, q))));
#pragma unroll
    for (int q = 0; q < 8; q++) e[q] = __reduce_max_sync(0xffffffffu, e[q]);
    long long a[8];
#pragma unroll
    for (int q = 0; q < 8; q++) a[q] = 0;
    for (int l = lane; l < n; l += 32)
#pragma unroll
        for (int q = 0; q < 8; q++) a[q] += fix_val(fix_counted(val(o + l, q)), e[q]);
    double t[NMOM];
#pragma unroll
    for (int q = 0; q < 8; q++) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], d);
        t[1 + q] = fix_total(a[q], e[q]);
    }
    if (lane == 0) {
        t[0] = n;
        t[9] = t[1] * y[0];
        t[10] = t[1] * y[1];
        t[11] = t[4] * y[2];
        for (int k = 0; k < NMOM; k++) mo[k] = t[k];
        const double tmean = (double)(N0 + 1) / (2.0 * N0) * dT;
        win[c] = N0 * (ub + share * dux + tmean * y[0]);
        win[ncell + c] = N0 * (vb + share * duy + tmean * y[1]);
        win[2 * ncell + c] = N0 * t[9];
        win[3 * ncell + c] = N0 * t[10];
        win[4 * ncell + c] = N0 * t[11];
        tgt[c] = 1.0;
        tgt[ncell + c] = tgt[2 * ncell + c] = tgt[3 * ncell + c] = 0.0;
    }
}

}  // namespace

cudaError_t launch_ocean_at_centres(int ncell, const Geom &g, const Phys<double> &P, double *oc, cudaStream_t st)
{
    k_ocean_at_centres<<<(ncell + 127) / 128, 128, 0, st>>>(ncell, g, P, oc);
    return cudaGetLastError();
}

cudaError_t launch_features(const double *mom, const double *tgt, int ncell, const Geom &g, const Phys<double> &P,
                            const Ctrl *ctrl, double dt, int N0, int n_t, const float *Ylag, const double *oc,
                            float *X, cudaStream_t st)
{
    k_features<<<(ncell + 127) / 128, 128, 0, st>>>(mom, tgt, ncell, g, P, ctrl, dt, ramp_mean_share(N0, n_t), Ylag,
                                                     oc, X);
    return cudaGetLastError();
}

cudaError_t launch_collect_targets(const double *mom0, const double *mom1, const double *win, int ncell, int N0,
                                   double dT, const int *is_closure, const float *Yuse, Ctrl *ctrl, float *Ylag,
                                   float *Y, const float *Yp, double floor_acc, float *nerr, int *age,
                                   cudaStream_t st)
{
    k_collect_targets<<<(ncell + 127) / 128, 128, 0, st>>>(mom0, mom1, win, ncell, N0, dT, is_closure, Yuse, ctrl,
                                                            Ylag, Y, Yp, floor_acc, nerr, age);
    return cudaGetLastError();
}

cudaError_t launch_hybrid_select(const HybridArgs &h, cudaStream_t st)
{
    k_classify<<<(h.ncell + 127) / 128, 128, 0, st>>>(h.X, h.Yp, h.mom, h.ncell, h.P64, h.rho_ice, h.box, h.tol,
                                                     h.mode, h.ctrl, h.nerr, h.age, h.is_closure, h.Yuse,
                                                     h.closure_count);
    if (h.nvgroups > 0)
        k_group_veto<<<(h.nvgroups + 127) / 128, 128, 0, st>>>(h.vgroups, h.nvgroups, h.vitems, h.off, h.is_closure,
                                                                h.closure_count);
    if (h.seg_mask) k_compact<<<h.nseg, 1024, 0, st>>>(h.order, h.seg_begin, h.seg_end, h.is_closure, h.order2, h.live,
                                                        h.seg_mask);
    k_closure_apply<<<(h.ncell + CA_WARPS - 1) / CA_WARPS, 32 * CA_WARPS, 0, st>>>(
        h.st32, h.P32, h.off, h.is_closure, h.Yuse, h.mom_rw, h.win, h.tgt, h.ncell, h.N0, h.dT,
        ramp_mean_share(h.N0, h.n_t));
    return cudaGetLastError();
}

}  // namespace msd
