// common.cuh -- types and device physics shared by the kernels of libmsdem.
//
// Physics follows Deng, Stechmann & Chen (arXiv 2303.07819):
//   DEM of disk floes, Sec. 2.1, Eq. (2.1a-d); contact law Eq. (2.2) with the
//   Coulomb limit; ocean (and wind) drag of Eq. (2.1c-d); forward Euler,
//   Sec. 3.1.  Readings of the places the paper leaves open are stated where
//   they are used.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msd {

constexpr int NMOM = 12;      // moment columns (see msdem.h)
constexpr int NWIN = 5;       // window columns
constexpr int MAXM = 16;      // stream-function modes
constexpr int NSUB_MAX = 8;   // Lax-Friedrichs substeps per coarse step (device-chosen N1)

// error bits raised by kernels, read by the host after a call
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_TIMEOUT = 2;
constexpr int ERR_CFL = 4;

// Device-resident control block of one model.
struct Ctrl {
    long long base;               // fine steps done before the current coarse interval (multiple of N0)
    int have_q;                   // coarse state initialised
    int have_tgt;                 // targets of the gradual update set
    int err;                      // ERR_* bits
    int N1;                       // LF substeps of the last coarse step
    unsigned int queue[2];        // work-queue tickets, one per step parity
    unsigned long long deep;      // contacts with overlap deeper than r_min / 2 (diagnostic)
    long long lag_mark;           // base + 1 at whose start the stored last-interval tendencies are valid
    unsigned int gq[3][2];        // group queues of the resident block kernels (ticket, blocks done), by class
    unsigned int pad[2];
};

// Physical constants in the kernel's arithmetic type.
//
// Ocean modes (stream-function modes first, then velocity modes): every mode
// m adds (-mAu, mAv) cos(th) to the current and -mAz sin(th) to its curl, th
// = mKx X + mKy Y + mPh.  A stream-function mode A sin(th) has (mAu, mAv,
// mAz) = (A ky, A kx, A |k|^2); a velocity mode (Au, Av) cos(th) has
// (-Au, Av, Av kx - Au ky).  FP64 kernels evaluate th directly.  FP32 kernels
// split th into the phase at the cell's corner (in cycles, reduced to [0, 1))
// and the turn across the cell: for a stream-function mode the wave numbers
// are integers per domain, so the corner phase is reduced exactly with the
// integer cell index; a velocity mode may have any real wave numbers, and its
// corner phase is reduced in FP64.
template <class R>
struct Phys {
    R uo_x, uo_y;
    int n_modes;                                   // stream-function + velocity modes
    R mA[MAXM], mKx[MAXM], mKy[MAXM], mPh[MAXM];   // A (stream modes), kx, ky (rad per length), phi
    R mAu[MAXM], mAv[MAXM], mAz[MAXM];             // see above
    R mAd[MAXM];                                   // divergence: -mAd sin(th) (Au kx + Av ky; 0 for stream modes)
    int isint[MAXM];                               // 1: stream mode with integer wave numbers per domain
    int mkx[MAXM], mky[MAXM];                      // FP32, integer modes: wave numbers per domain
    R mCyc[MAXM];                                  // FP32: phi / 2 pi reduced to [0, 1)
    double bx[MAXM], by[MAXM], bph[MAXM];          // FP32, real modes: cycles per cell in x, y, phi / 2 pi (FP64)
    R kcx[MAXM], kcy[MAXM];                        // FP32, real modes: the same in FP32 (turn across a cell)
    R kdx[MAXM], kdy[MAXM];                        // FP32: cycles per domain (the truth DEM's phase)
    int taylor;                                    // FP32: 1 if every mode turns by <= 1/16 cycle across a cell
    R ocean_d2;                                    // FP32 (variant 5): squared distance (m^2) a floe may move from
                                                   // the centre of its local ocean expansion (see cell_run.cu)
    R ta[MAXM], tb[MAXM];                          // FP32: kx Lcx, ky Lcy (radians per cell)
    R drag_o;      // Cd rho_o pi
    R drag_a;      // Ca rho_a pi
    R wind_x, wind_y, wind_w;   // wind at t = 0 and its turning rate 2 pi / period
    R mass_c;      // rho_ice pi
    R inertia_f;   // 1 (paper) or 1/2
    R E, G, eta, mu, inv_h_ref;
};

// Coarse grid.  An ensemble of nens independent realizations is stored as
// nens copies of the nx x nyr grid stacked in y (ny = nens nyr rows, Ly =
// nens times one realization's side); each realization is periodic on its own.
struct Geom {
    int nx, ny;
    double Lx, Ly, Lcx, Lcy;
    int nyr, nens;      // rows per realization, realizations
    int walls;          // 1, 2: rigid walls at x = 0 and x = Lx (Sec. 4.4); 0: periodic in x
};

// ---------------------------------------------------------------- helpers
template <class R> __device__ __forceinline__ R dmin(R a, R b) { return a < b ? a : b; }
template <class R> __device__ __forceinline__ R dmax(R a, R b) { return a > b ? a : b; }

// 1/sqrt(x): the hardware reciprocal square root in FP32, the IEEE
// operations in FP64 (the parity path)
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }

// Contact of floe l with floe j given the minimum-image separation
// (dx, dy) = x_j - x_l.  Eq. (2.2): n from l to j, delta = d - (r_l + r_j) < 0
// in overlap; normal force c h (E delta + eta v_n) n, never attractive
// (reading: optional dashpot eta; thickness factor h = min(h_l, h_j)/h_ref);
// tangential c h G v_t t with |f_t| <= mu |f_n|; torque r_l f_t on l.
// The chord c of the overlap lens is written symmetrically in (l, j):
// c^2 d^2 = (S - d)(S + d)(d - D)(d + D), S = r_l + r_j, D = r_l - r_j
// (Heron's formula for the triangle (d, r_l, r_j)); a floe inside the other
// (d <= |D|) gives the smaller diameter.
// Returns true on contact and adds the force on l to (fx, fy, tq).
template <class R>
__device__ __forceinline__ bool contact_add(R dx, R dy, R d2, R rl, R rj, R hl, R hj,
                                            R dux, R duy, R wl, R wj, const Phys<R> &P,
                                            R &fx, R &fy, R &tq, unsigned &deep)
{
    const R S = rl + rj;
    if (!(d2 > R(0) && d2 < S * S)) return false;
    const R id = inv_sqrt(d2);
    const R d = d2 * id;
    const R nx = dx * id, ny = dy * id;
    const R delta = d - S;
    const R D = rl - rj;
    const R Q = (d - D) * (d + D);
    const R c = (Q <= R(0)) ? R(2) * dmin(rl, rj) : sqrt((-delta) * (S + d) * Q) * id;
    const R hc = dmin(hl, hj) * P.inv_h_ref;
    const R vn = dux * nx + duy * ny;
    R Fn = c * hc * (P.E * delta + P.eta * vn);
    Fn = dmin(Fn, R(0));
    const R vt = dux * (-ny) + duy * nx - wj * rj - wl * rl;
    R ft = c * hc * P.G * vt;
    const R cap = P.mu * (-Fn);
    ft = dmax(dmin(ft, cap), -cap);
    fx += Fn * nx - ft * ny;
    fy += Fn * ny + ft * nx;
    tq += rl * ft;
    deep |= (delta < R(-0.5) * dmin(rl, rj)) ? 1u : 0u;
    return true;
}

// Ocean drag at the floe plus wind drag, Eq. (2.1c-d): translation
// alpha (u - v)|u - v| with alpha = Cd rho_o pi r^2 (wind: Ca rho_a pi r^2),
// rotation beta (zeta/2 - w)|zeta/2 - w| with beta = Cd rho_o pi r^4.
template <class R>
__device__ __forceinline__ void drag_force(const Phys<R> &P, R uo, R vo, R zeta, R ua, R va,
                                           R u, R v, R w, R r, R &Fx, R &Fy, R &T)
{
    const R ao = P.drag_o * r * r;
    const R aa = P.drag_a * r * r;
    const R bo = P.drag_o * r * r * r * r;
    const R du = uo - u, dv = vo - v;
    const R so = sqrt(du * du + dv * dv);
    const R au = ua - u, av = va - v;
    const R sa = sqrt(au * au + av * av);
    const R dw = R(0.5) * zeta - w;
    Fx = ao * du * so + aa * au * sa;
    Fy = ao * dv * so + aa * av * sa;
    T = bo * dw * fabs(dw);
}

// Ocean current and its curl at a global position, FP64 (mode coefficients
// as described at Phys).
__device__ __forceinline__ void ocean_f64(const Phys<double> &P, double X, double Y,
                                          double &uo, double &vo, double &zeta)
{
    uo = P.uo_x; vo = P.uo_y; zeta = 0.0;
    for (int m = 0; m < P.n_modes; m++) {
        const double th = P.mKx[m] * X + P.mKy[m] * Y + P.mPh[m];
        double s, c;
        sincos(th, &s, &c);
        uo -= P.mAu[m] * c;
        vo += P.mAv[m] * c;
        zeta -= P.mAz[m] * s;
    }
}

// Divergence of the current at a global position, FP64.
__device__ __forceinline__ double ocean_div_f64(const Phys<double> &P, double X, double Y)
{
    double d = 0.0;
    for (int m = 0; m < P.n_modes; m++)
        if (P.mAd[m] != 0.0) d -= P.mAd[m] * sin(P.mKx[m] * X + P.mKy[m] * Y + P.mPh[m]);
    return d;
}

// FP32 phase of mode m at the corner of cell (ix, iy), in cycles, in [0, 1]:
// ((kx ix) mod nx)/nx + ((ky iy) mod ny)/ny + phi/2pi with the integer part
// reduced exactly (stream modes), or the FP64 product reduced (real modes).
__device__ __forceinline__ float corner_phase(const Phys<float> &P, int m, int ix, int iy, int nx, int ny,
                                              float inx, float iny)
{
    if (P.isint[m]) {
        int ax = (P.mkx[m] * ix) % nx; if (ax < 0) ax += nx;
        int ay = (P.mky[m] * iy) % ny; if (ay < 0) ay += ny;
        const float b = (float)ax * inx + (float)ay * iny + P.mCyc[m];
        return b - floorf(b);
    }
    double b = P.bx[m] * ix + P.by[m] * iy + P.bph[m];
    return (float)(b - floor(b));
}

// FP32 turn of mode m across the fraction (xf, yf) of a cell, in cycles
__device__ __forceinline__ float turn_x(const Phys<float> &P, int m, float xf, float inx)
{
    return P.isint[m] ? (float)P.mkx[m] * xf * inx : P.kcx[m] * xf;
}
__device__ __forceinline__ float turn_y(const Phys<float> &P, int m, float yf, float iny)
{
    return P.isint[m] ? (float)P.mky[m] * yf * iny : P.kcy[m] * yf;
}

// FP32 ocean at cell (ix, iy) + fraction (xf, yf) of the cell; base[m] is the
// mode's corner phase (corner_phase).
__device__ __forceinline__ void ocean_f32(const Phys<float> &P, const float *base, float inx,
                                          float iny, float xf, float yf, float &uo, float &vo,
                                          float &zeta)
{
    uo = P.uo_x; vo = P.uo_y; zeta = 0.0f;
    for (int m = 0; m < P.n_modes; m++) {
        const float cyc = base[m] + turn_x(P, m, xf, inx) + turn_y(P, m, yf, iny);
        float s, c;
        sincospif(2.0f * cyc, &s, &c);
        uo -= P.mAu[m] * c;
        vo += P.mAv[m] * c;
        zeta -= P.mAz[m] * s;
    }
}

// Wind vector at time t: the t = 0 vector turned by wind_w * t.
template <class R>
__device__ __forceinline__ void wind_at(const Phys<R> &P, double t, R &ua, R &va)
{
    if (P.wind_w != R(0)) {
        double s, c;
        sincos((double)P.wind_w * t, &s, &c);
        ua = (R)((double)P.wind_x * c - (double)P.wind_y * s);
        va = (R)((double)P.wind_x * s + (double)P.wind_y * c);
    } else {
        ua = P.wind_x;
        va = P.wind_y;
    }
}

// ------------------------------------------------------ launch interfaces
struct DevState32 {
    uint32_t *xq, *yq;
    float *th, *u, *v, *w, *r, *h;
};
struct DevState64 {
    double *x, *y, *th, *u, *v, *w, *r, *h;
};

constexpr int MAXSEG = 10;   // size classes of cells launched separately (binned variants)

struct CellLaunch {
    int variant;       // 0 brute force, 1 binned block per cell, 2 binned warp per cell, 3 as 2 with
                       // the warp classes resident for a run of steps (FP32 only)
    int threads;       // threads per block (brute force)
    float bin_beta;    // bin side in units of the mean floe spacing (binned variant)
    int persistent;    // 1: grid of resident blocks + work queue (brute force)
    int grid;          // blocks for the persistent form
    // binned variant: cells in processing order split into size classes, each
    // launched with its own block size and shared memory
    int nseg;
    int seg_begin[MAXSEG], seg_end[MAXSEG], seg_maxn[MAXSEG], seg_threads[MAXSEG];
    int seg_kind[MAXSEG];   // 0: block per cell, 1: warp per cell (seg_maxn = the warp's capacity),
                            // 2: cells of <= 32 floes packed several to a warp, 3: resident
                            // blocks, seg_maxn / 256 floes per thread (variant 5)
    const int2 *pack;  // kind 2: per warp (first item, cells), device
    int npack;
    int nbmax;         // bins per side at most
    // variant 5, kind 3 segments (resident block classes): per segment the
    // groups of cells one block takes (device) and their number; per group
    // slot the cell and its place in the group (device)
    const int4 *rgroups[MAXSEG];
    int rngroups[MAXSEG];
    const int4 *ritems;
    float run_skin;    // variant 5: horizon of a floe's skin, fine steps at its build speed
    int run_cap1;      // variant 5: floes per block of small cells (at most RUN_T)
    // segments of variant 2 run on their own streams, forked from and joined
    // back into the launching stream (concurrent branches in a graph)
    cudaStream_t side[MAXSEG];
    cudaEvent_t ev_fork, ev_join[MAXSEG];
};

// FP32 constants of a launch, computed once on the host (FP64 arithmetic on
// the device runs at a small fraction of the FP32 rate).
struct Geo32 {
    float sx, sy;       // cell side / 2^32 (fixed point -> m)
    float isx, isy;     // 2^32 / cell side
    float inx, iny;     // 1 / nx, 1 / ny
    float Lx, Ly;       // cell sides (m)
    float iLx, iLy;
    float dt;
};

// Contact candidate lists of the FP32 state (variant 4): per floe up to NBL
// cell-local floe indices in search order.  The count and the first NLH
// entries share one 16-byte head, so a floe's list starts with one load; the
// rest follow in 16-byte groups of 8 entries, floe-major.  Also the positions
// the lists were built from, and per cell the step of the build (< 0: none)
// and the skin.
constexpr int NLH = 7;               // entries in the head
constexpr int NLT = 3;               // 8-entry tail groups per floe
constexpr int NBL = NLH + 8 * NLT;   // candidate list entries per floe

struct NbLists {
    uint4 *head;        // [n]: 16-bit halves: count, then entries 0 .. NLH-1
    uint4 *tail;        // [n][NLT]: entries NLH .. NBL-1, 8 per group
    uint2 *xb;          // [n] fixed-point position at the build
    long long *cstep;   // [ncell]
    float *skin;        // [ncell]
};

struct StepCommon {
    Geo32 k;
    NbLists nl;         // candidate lists of the state the launch writes
    const int *live;    // per size class: cells to step (the rest run the closure); nullptr: all
    const int *off;     // [ncell + 1]
    const int *order;   // [ncell] processing order (largest cells first); in closure mode the
                        // particle cells of each size class first
    const int *order0;  // [ncell] processing order (the packed warps' table refers to it)
    const int *skip;    // [ncell] 1: the cell runs the closure this interval (packed warps); nullptr: none
    int ncell;
    int max_n;          // largest cell
    double *mom;        // [ncell][NMOM]
    double *win;        // [NWIN][ncell]
    const double *tgt;  // [4][ncell]
    Ctrl *ctrl;
    Geom g;
    double dt;
    int N0, n_t, couple;
    long long i_local;  // step within the current coarse interval (0-based)
    // variant 5: what a run hands to the next, [RUN_NCARRY][ncarry]: the
    // floes' running window sums (velocity u, v, drag Fx, Fy, torque since
    // the last gradual update) and the fixed-point centre of each floe's
    // ocean expansion; read at a run that starts inside an interval, written
    // by one that ends inside one
    const float *carry_in;
    float *carry_out;
    long long ncarry;
};

// 2^32 and 2^-32: fixed-point positions of the FP32 path (2^32 = cell side)
constexpr float TWO32F = 4294967296.0f;
constexpr float INV2_32F = 2.3283064365386963e-10f;

// e^{i th} for |th| <= 0.4 by its Taylor series to th^9 (error < 1e-10)
__device__ __forceinline__ void rot_small(float th, float &c, float &s)
{
    const float t = th * th;
    c = fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
    s = th * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
}

// Gradual update of one cell (Sec. 3.3, Eqs. 3.5-3.7).  reading: each update
// adds n_t/N0 of (target - snapshot at the coarse step); radii follow
// r = r0 (1 + (s - 1) ev n_t/N0), applied as the per-step ratio g.
struct RampCell {
    double g, du, dv, dw;
};

__device__ __forceinline__ RampCell ramp_cell(const StepCommon &sc, int c, int ev)
{
    const int nc = sc.ncell;
    const double f = (double)sc.n_t / (double)sc.N0;
    const double s = sc.tgt[c];
    RampCell rc;
    rc.g = (1.0 + (s - 1.0) * ev * f) / (1.0 + (s - 1.0) * (ev - 1) * f);
    rc.du = sc.tgt[nc + c] * f;
    rc.dv = sc.tgt[2 * nc + c] * f;
    rc.dw = sc.tgt[3 * nc + c] * f;
    return rc;
}

constexpr int RUN_T = 256;      // threads per block of the resident block kernels (variant 5)
constexpr int RUN_GCMAX = 32;   // cells per group of those kernels
constexpr int RUN_NCARRY = 7;   // words per floe a run hands to the next: 5 window sums, ocean expansion centre

// cell_run.cu: a run of nsteps fine steps of one block class (K floes per
// thread) from step sc.i_local of the interval, every floe in registers
// (launch variant 5).  groups[g] = (first slot, cells, floes, bins incl. one
// large-floe slot per cell) in processing order; items[slot] = (cell, first
// floe of the cell in its group, bins per side (0: none), bin base); the
// carry is sc.carry_in / sc.carry_out; qslot = the class's queue in Ctrl.
cudaError_t launch_run_block(int K, const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                             const StepCommon &sc, const int4 *groups, int ngroups, const int4 *items, int qslot,
                             int nsteps, float skin_steps, cudaStream_t st);
size_t run_block_smem(int K);
cudaError_t run_block_prepare();
// fold the running window sums of a run that stopped inside a coarse interval
// into the window (masses of the current state) and clear them
cudaError_t launch_carry_flush(const DevState32 &s, const StepCommon &sc, float *carry, long long ncarry,
                               cudaStream_t st);

// cell_step.cu
cudaError_t launch_cell_step32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                               const StepCommon &sc, const CellLaunch &cl, cudaStream_t st);
// nsteps fine steps of every size class from step sc.i_local of the interval,
// each class on its own stream (variants 2 and 3; the streams forked by
// cell_fork); variant 3 runs each warp class's steps in one resident launch
cudaError_t launch_cell_run32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                              const StepCommon &sc, const CellLaunch &cl, int nsteps);
// fork the size-class streams off st / join them back (variants 2 and 3)
cudaError_t cell_fork(const CellLaunch &cl, cudaStream_t st);
cudaError_t cell_join(const CellLaunch &cl, cudaStream_t st);
cudaError_t launch_cell_step64(const DevState64 &in, const DevState64 &out, const Phys<double> &P,
                               const StepCommon &sc, const CellLaunch &cl, cudaStream_t st);
cudaError_t launch_cell_moments32(const DevState32 &s, const Phys<float> &P, const StepCommon &sc,
                                  cudaStream_t st);
cudaError_t launch_cell_moments64(const DevState64 &s, const Phys<double> &P, const StepCommon &sc,
                                  cudaStream_t st);
size_t cell_step_smem(int precision, const CellLaunch &cl, int max_n, int nx, int ny);
int seg_nbmax(const CellLaunch &cl, int s);
cudaError_t cell_step_prepare(int precision, const CellLaunch &cl, size_t smem);

// coarse.cu
struct CoarseArgs {
    int nx, ny;         // ny: rows of all realizations
    int nyr, nens;      // rows per realization, realizations
    int walls;          // ghost cells beyond x = 0 and x = Lx (Sec. 4.4): 1 zero, 2 mirrored
    unsigned long long *cmax;   // [nens] max over the realization's cells of |V|/dx (non-negative double bits)
    double dx, dy, Ac, dT;
    int N0;
    const double *mom;  // [ncell][NMOM]
    double *win;        // [NWIN][ncell]
    double *q0, *q1;    // [4][ncell] ping-pong
    double *V;          // [2][ncell]
    double *S;          // [4][ncell]
    double *tgt;        // [4][ncell]
    Ctrl *ctrl;
};
cudaError_t launch_coarse_step(const CoarseArgs &a, cudaStream_t st);   // one cooperative launch
cudaError_t fma_probe(int reps, double *tflops);                          // probe.cu
cudaError_t launch_advance(Ctrl *ctrl, int N0, cudaStream_t st);       // base += N0
int coarse_launches();

// truth.cu
// Bins of the truth DEM (and of the per-cell moment binning): floes of radius
// <= r_split in a grid of nbx x nby bins, the others in a second grid of
// nbx2 x nby2 bins (0 x 0: none), one bin index space (the second grid's bins
// after the first's).
struct TruthBins {
    int nbx, nby;          // bins per side (1 x 1: brute force)
    int nbx2, nby2;        // the large floes' grid
    float r_split;
    __host__ __device__ int nbins() const { return nbx * nby + nbx2 * nby2; }
    int *count;            // [nbins]
    int *start;            // [nbins + 1]
    int *cursor;           // [nbins]
    int *sorted;           // [n] floe indices grouped by bin
    int *bin;              // [n]
    int *scan_tmp;         // block sums
    int nscan_blocks;
};
struct TruthArgs {
    long long n;
    Geom g;
    Geo32 k;               // domain-sized constants (fixed point of the domain)
    double dt;
    long long step;        // steps done before this one
    Ctrl *ctrl;            // error bits and deep-overlap counter
    void *fd;              // [3][n] drag of the last step (R)
};
cudaError_t launch_truth_step32(const DevState32 &in, const DevState32 &out, const Phys<float> &P,
                                const TruthArgs &a, TruthBins &b, cudaStream_t st);
cudaError_t launch_truth_step64(const DevState64 &in, const DevState64 &out, const Phys<double> &P,
                                const TruthArgs &a, TruthBins &b, cudaStream_t st);
cudaError_t launch_truth_moments32(const DevState32 &s, const Phys<float> &P, const TruthArgs &a,
                                   TruthBins &cells, double *mom, cudaStream_t st);
cudaError_t launch_truth_moments64(const DevState64 &s, const Phys<double> &P, const TruthArgs &a,
                                   TruthBins &cells, double *mom, cudaStream_t st);
int truth_launches(const TruthBins &b);
// per-cell moments with scratch from a static device array (no allocation)
long long noalloc_max_floes();
int noalloc_max_cells();
cudaError_t noalloc_cell_moments(const Geom &g, double mass_c, double inertia_f, long long n, const double *x,
                                 const double *y, const double *u, const double *v, const double *w,
                                 const double *r, const double *h, const double *fd, double *mom,
                                 cudaStream_t st);
cudaError_t bins_scan(TruthBins &b, int nbins, cudaStream_t st);

// hybrid.cu: closure-plus-fallback intervals
struct HybridArgs {
    const float *X;           // features [ncell][NFEAT]
    float *Yp;                // network prediction [ncell][4] (mode 2: made absolute in place)
    const float *nerr;        // [ncell] the network's drag error on the cell's last DEM interval
    const int *age;           // [ncell] closure intervals since that DEM interval
    const double *mom;
    int ncell, nseg;
    Phys<double> P64;
    Phys<float> P32;
    double rho_ice, tol, floor_acc, dT;
    const float *box;         // [2][NFEAT] feature range seen in training
    int mode;                 // 0 network, 1 mean-field
    const Ctrl *ctrl;
    int *is_closure;
    float *Yuse;
    const int *order, *seg_begin, *seg_end, *off;
    int *order2, *live;
    unsigned long long *closure_count;
    unsigned seg_mask;        // classes whose particle cells are compacted into order2 / live
    // groups of cells that share a block for a whole interval (resident
    // kernels): a cell keeps the closure only if every cell with floes in its
    // group does (device; nvgroups = 0: none)
    const int4 *vgroups, *vitems;
    int nvgroups;
    DevState32 st32;
    double *win, *tgt;
    double *mom_rw;
    int N0, n_t;
};
constexpr int NFEAT = 16;   // closure features per cell (12 from the moments and forcing, 4 lagged tendencies)
// oc = [ncell][4] ocean u, v, divergence and curl at the cell centres
cudaError_t launch_ocean_at_centres(int ncell, const Geom &g, const Phys<double> &P, double *oc, cudaStream_t st);
cudaError_t launch_features(const double *mom, const double *tgt, int ncell, const Geom &g, const Phys<double> &P,
                            const Ctrl *ctrl, double dt, int N0, int n_t, const float *Ylag, const double *oc,
                            float *X, cudaStream_t st);
cudaError_t launch_collect_targets(const double *mom0, const double *mom1, const double *win, int ncell, int N0,
                                   double dT, const int *is_closure, const float *Yuse, Ctrl *ctrl, float *Ylag,
                                   float *Y, const float *Yp, double floor_acc, float *nerr, int *age,
                                   cudaStream_t st);
// closure intervals a cell may run between two DEM intervals that check the network on it
constexpr int CLOSURE_MAX_RUN = 3;
cudaError_t launch_hybrid_select(const HybridArgs &h, cudaStream_t st);

// api.cu: record the calling thread's error message and return code
int set_error(int code, const char *msg);

}  // namespace msd
