// api.cu -- host side of libmsdem: validation, device layout, the
// Algorithm 1 schedule (fine steps, coarse steps, gradual updates) captured
// in CUDA graphs, the truth DEM driver, and the C-ABI of include/msdem.h.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "classes.cuh"
#include "common.cuh"
#include "shard.cuh"
#include "upload.cuh"
#include "../../include/msdem.h"

using namespace msd;

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int msd::set_error(int code, const char *msg) { return fail(code, "%s", msg); }

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(MS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

static const double PI_D = 3.14159265358979323846;

// NVTX range over a host-side phase (API call, graph replay, coarse step):
// profilers attribute the kernels launched inside it to the phase; without a
// profiler attached the calls cost next to nothing.
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};

struct ms_model {
    int precision = 0;
    ms_grid grid{};
    ms_forcing fc{};
    std::vector<double> modes, vmodes;
    long long n = 0;
    int ncell = 0, max_n = 0;
    Geom g{};
    Phys<float> P32{};
    Phys<double> P64{};
    // layout: stored floe k of cell c at off[c] + ...; orig[k] = caller's index
    std::vector<int> h_off, h_order, h_cell_of_orig;
    std::vector<long long> h_orig;
    int *d_off = nullptr, *d_order = nullptr;
    // uploads: the caller's arrays as sent ([8][n] FP64), orig and cell of
    // the caller's floes on the device, the checks' first failing indices
    double *d_raw = nullptr;
    int *d_orig = nullptr, *d_cell_of = nullptr;
    unsigned long long *d_first = nullptr;
    // msDEM state and its scratch copy for out-of-place timing
    DevState32 s32{}, x32{};
    NbLists nl{}, xnl{};          // candidate lists of s32 and of the timing copy x32
    DevState64 s64{}, x64{};
    double *d_mom = nullptr, *d_win = nullptr, *d_q0 = nullptr, *d_q1 = nullptr, *d_V = nullptr,
           *d_S = nullptr, *d_tgt = nullptr, *d_xmom = nullptr, *d_xwin = nullptr;
    Ctrl *d_ctrl = nullptr;
    unsigned long long *d_cmax = nullptr;   // [nens] coarse-step CFL maxima
    int2 *d_pack = nullptr;                  // [ncell] packed-warp table (at most one warp per cell)
    int4 *d_rgroups = nullptr, *d_ritems = nullptr;   // [ncell] variant 5: groups of cells per block, cell places
    float *d_carry = nullptr, *d_xcarry = nullptr;    // [RUN_NCARRY][n] variant 5: what a run hands to the next
    // truth
    DevState32 t32[2]{};
    DevState64 t64[2]{};
    int tcur = 0;
    void *d_fd = nullptr;
    TruthBins tb{}, cb{};
    double *d_tmom = nullptr;
    // schedule
    long long steps = 0, truth_steps = 0;
    double dt = 0.0, truth_dt = 0.0;
    int interval = 100;   // steps per coarse interval (graph length)
    cudaStream_t stream = nullptr, own_stream = nullptr, side_stream[MAXSEG] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[MAXSEG] = {};
    CellLaunch cl{};
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
    long long replays = 0;
    int sm_count = 0;
    // closure-plus-fallback intervals
    ms_mlp *mlp = nullptr;
    int hybrid_mode = -1;          // -1 off, 0 network, 1 mean-field
    double hybrid_tol = 0.0;
    float *d_X = nullptr, *d_Yp = nullptr, *d_Yuse = nullptr, *d_box = nullptr, *d_Yc = nullptr, *d_Ylag = nullptr,
          *d_nerr = nullptr;
    int *d_age = nullptr;
    int *d_isc = nullptr, *d_order2 = nullptr, *d_live = nullptr, *d_segb = nullptr, *d_sege = nullptr;
    double *d_mom0 = nullptr;
    double *d_ocean = nullptr;      // [ncell][4] ocean at the cell centres (closure features)
    unsigned long long *d_ccount = nullptr;
    long long hybrid_intervals = 0;
    // a grid split into tiles: this model holds the floes of cells
    // shard_cells[0 .. shard_nown) (device copy: the cells of every rank, in
    // rank order, and their rows of the gathered buffer)
    int shard_nranks = 0, shard_rank = 0, shard_nown = 0, shard_maxc = 0, shard_first = 0;
    int *d_shard_cells = nullptr;
    long long *d_shard_rows = nullptr;
    double *d_send = nullptr, *d_recv = nullptr;
    ms_exchange_fn exch = nullptr;
    void *exch_ctx = nullptr;
    bool exch_failed = false;
    cudaGraphExec_t gexec_end = nullptr;   // sharded: the interval's coarse step after the exchange
    // host staging (pinned)
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    std::vector<void *> allocs;
};

// ---------------------------------------------------------------- helpers
template <class T>
static cudaError_t dalloc(ms_model *m, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count > 0 ? count : 1));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return cudaSuccess;
}

static cudaError_t alloc32(ms_model *m, DevState32 &s, size_t n)
{
    cudaError_t e;
    if ((e = dalloc(m, &s.xq, n)) || (e = dalloc(m, &s.yq, n)) || (e = dalloc(m, &s.th, n)) ||
        (e = dalloc(m, &s.u, n)) || (e = dalloc(m, &s.v, n)) || (e = dalloc(m, &s.w, n)) ||
        (e = dalloc(m, &s.r, n)) || (e = dalloc(m, &s.h, n)))
        return e;
    return cudaSuccess;
}

static cudaError_t alloc_lists(ms_model *m, NbLists &l, size_t n, int ncell)
{
    cudaError_t e;
    if ((e = dalloc(m, &l.head, n)) || (e = dalloc(m, &l.tail, n * NLT)) || (e = dalloc(m, &l.xb, n)) ||
        (e = dalloc(m, &l.cstep, ncell)) || (e = dalloc(m, &l.skin, ncell)))
        return e;
    return cudaMemsetAsync(l.cstep, 0xff, sizeof(long long) * ncell, m->stream);
}

// forget the candidate lists (the floes changed outside a cell step)
static cudaError_t invalidate_lists(ms_model *m)
{
    cudaError_t e = cudaSuccess;
    if (m->nl.cstep) e = cudaMemsetAsync(m->nl.cstep, 0xff, sizeof(long long) * m->ncell, m->stream);
    if (e == cudaSuccess && m->xnl.cstep)
        e = cudaMemsetAsync(m->xnl.cstep, 0xff, sizeof(long long) * m->ncell, m->stream);
    return e;
}

static cudaError_t alloc64(ms_model *m, DevState64 &s, size_t n)
{
    cudaError_t e;
    if ((e = dalloc(m, &s.x, n)) || (e = dalloc(m, &s.y, n)) || (e = dalloc(m, &s.th, n)) ||
        (e = dalloc(m, &s.u, n)) || (e = dalloc(m, &s.v, n)) || (e = dalloc(m, &s.w, n)) ||
        (e = dalloc(m, &s.r, n)) || (e = dalloc(m, &s.h, n)))
        return e;
    return cudaSuccess;
}

// Pinned host staging buffer.  Copies from and to it are asynchronous, so
// every use first waits for the model's stream: a previous upload may still
// be reading it.
static void *stage(ms_model *m, size_t bytes)
{
    if (m->stream && cudaStreamSynchronize(m->stream) != cudaSuccess) return nullptr;
    if (bytes > m->h_stage_bytes) {
        if (m->h_stage) cudaFreeHost(m->h_stage);
        m->h_stage = nullptr;
        m->h_stage_bytes = 0;
        if (cudaMallocHost(&m->h_stage, bytes) != cudaSuccess) return nullptr;
        m->h_stage_bytes = bytes;
    }
    return m->h_stage;
}

static bool isfin(double x) { return std::isfinite(x); }

// the model's geometry of a grid (an ensemble stacks its realizations in y)
static Geom grid_geom(const ms_grid *grid)
{
    const int nens = grid->nens > 1 ? grid->nens : 1;
    Geom g{};
    g.nx = grid->nx;
    g.ny = grid->ny * nens;
    g.nyr = grid->ny;
    g.nens = nens;
    g.Lx = grid->Lx;
    g.Ly = grid->Ly * nens;
    g.Lcx = grid->Lx / grid->nx;
    g.Lcy = grid->Ly / grid->ny;
    g.walls = grid->walls;
    return g;
}

static uint32_t to_fix(double frac)
{
    // fraction of the periodic box -> 32-bit fixed point (2^32 == 1, wraps)
    double v = std::nearbyint(frac * 4294967296.0);
    long long iv = (long long)v;
    return (uint32_t)(iv & 0xffffffffLL);
}

static double from_fix(uint32_t q) { return (double)q * (1.0 / 4294967296.0); }

// f(begin, end) over [0, n) in contiguous chunks on the host's cores (the
// per-floe loops of uploads, downloads and their checks; each index is
// handled by exactly one chunk, so the results do not depend on the split)
template <class F>
static void host_parallel(long long n, F &&f)
{
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt == 0 ? 1u : (nt > 32u ? 32u : nt);
    if (n < 65536 || nt == 1) {
        f(0LL, n);
        return;
    }
    const long long chunk = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; t++) {
        const long long b = t * chunk, e = std::min(n, b + chunk);
        if (b < e) th.emplace_back([&f, b, e] { f(b, e); });
    }
    f(0LL, std::min(n, chunk));
    for (auto &x : th) x.join();
}

// smallest index in [0, n) for which bad(l) holds, or n
template <class B>
static long long host_first(long long n, B &&bad)
{
    std::atomic<long long> first{LLONG_MAX};
    host_parallel(n, [&](long long b, long long e) {
        for (long long l = b; l < e; l++)
            if (bad(l)) {
                long long cur = first.load();
                while (l < cur && !first.compare_exchange_weak(cur, l)) {
                }
                break;
            }
    });
    const long long f = first.load();
    return f < n ? f : n;
}

// the checks that need no per-floe pass: pointers and counts
static int check_floe_args(const ms_floes *f, long long expect_n)
{
    if (!f) return fail(MS_ERR_ARG, "floes is NULL");
    if (f->n < 0) return fail(MS_ERR_ARG, "floes->n = %lld < 0", (long long)f->n);
    if (expect_n >= 0 && f->n != expect_n)
        return fail(MS_ERR_ARG, "floes->n = %lld, model has %lld floes", (long long)f->n, expect_n);
    if (f->n > 0 && (!f->x || !f->y || !f->theta || !f->u || !f->v || !f->omega || !f->r || !f->h))
        return fail(MS_ERR_ARG, "a floe array is NULL");
    if (f->n > (long long)0x7fffffff) return fail(MS_ERR_ARG, "more than 2^31-1 floes");
    return MS_OK;
}

static bool floe_finite(const ms_floes *f, long long l)
{
    return isfin(f->x[l]) && isfin(f->y[l]) && isfin(f->theta[l]) && isfin(f->u[l]) && isfin(f->v[l]) &&
           isfin(f->omega[l]) && isfin(f->r[l]) && isfin(f->h[l]);
}

static int validate_floes(const ms_floes *f, long long expect_n)
{
    const int rc = check_floe_args(f, expect_n);
    if (rc) return rc;
    const long long l = host_first(f->n, [&](long long k) {
        return !floe_finite(f, k) || !(f->r[k] > 0.0) || !(f->h[k] > 0.0);
    });
    if (l < f->n) {
        if (!floe_finite(f, l)) return fail(MS_ERR_ARG, "floe %lld has a non-finite value", l);
        return fail(MS_ERR_ARG, "floe %lld has r <= 0 or h <= 0", l);
    }
    return MS_OK;
}

static UpGeom up_geom(const ms_model *m)
{
    UpGeom g;
    g.n = m->n;
    g.nx = m->g.nx;
    g.ny = m->g.ny;
    g.Lx = m->g.Lx;
    g.Ly = m->g.Ly;
    g.Lcx = m->g.Lcx;
    g.Lcy = m->g.Lcy;
    return g;
}

// the caller's eight arrays into the pinned stage (all host cores), then to
// the device's raw copy in one transfer (queued on the model's stream)
// true if p lies in page-locked host memory of this process (cudaHostAlloc,
// cudaHostRegister)
static bool host_pinned(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// the caller's eight floe arrays into d_raw on the model's stream: straight
// from the caller's memory when every array is page-locked, else through the
// pinned staging buffer array by array (the transfer of one array overlaps
// the host copy of the next)
static int send_raw(ms_model *m, const ms_floes *f)
{
    const long long n = m->n;
    const double *src[8] = {f->x, f->y, f->theta, f->u, f->v, f->omega, f->r, f->h};
    bool pinned = true;
    for (int a = 0; a < 8 && pinned; a++) pinned = host_pinned(src[a]);
    if (pinned) {
        for (int a = 0; a < 8; a++)
            CK(cudaMemcpyAsync(m->d_raw + a * n, src[a], sizeof(double) * n, cudaMemcpyHostToDevice, m->stream));
        return MS_OK;
    }
    double *st = (double *)stage(m, sizeof(double) * 8 * n);
    if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost of %lld bytes failed", (long long)(64 * n));
    for (int a = 0; a < 8; a++) {
        host_parallel(n, [&](long long k0, long long k1) {
            std::memcpy(st + a * n + k0, src[a] + k0, sizeof(double) * (k1 - k0));
        });
        CK(cudaMemcpyAsync(m->d_raw + a * n, st + a * n, sizeof(double) * n, cudaMemcpyHostToDevice, m->stream));
    }
    return MS_OK;
}

// the raw copy (already checked and assigned to cells) into the msDEM layout
static int raw_to_state(ms_model *m)
{
    if (m->n == 0) return MS_OK;
    const UpGeom g = up_geom(m);
    if (m->precision == MS_FP64)
        CK(launch_floes_to_cells64(m->d_raw, m->d_orig, m->d_cell_of, g, m->s64, m->stream));
    else
        CK(launch_floes_to_cells32(m->d_raw, m->d_orig, m->d_cell_of, g, m->s32, m->stream));
    return MS_OK;
}

static int upload_truth_state(ms_model *m, const ms_floes *f)
{
    const long long n = m->n;
    if (n == 0) return MS_OK;
    if (m->precision == MS_FP64) {
        double *st = (double *)stage(m, sizeof(double) * 8 * n);
        if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
        for (long long l = 0; l < n; l++) {
            st[l] = f->x[l] - m->g.Lx * std::floor(f->x[l] / m->g.Lx);
            st[n + l] = f->y[l] - m->g.Ly * std::floor(f->y[l] / m->g.Ly);
            st[2 * n + l] = f->theta[l];
            st[3 * n + l] = f->u[l];
            st[4 * n + l] = f->v[l];
            st[5 * n + l] = f->omega[l];
            st[6 * n + l] = f->r[l];
            st[7 * n + l] = f->h[l];
        }
        DevState64 &s = m->t64[m->tcur];
        double *dst[8] = {s.x, s.y, s.th, s.u, s.v, s.w, s.r, s.h};
        for (int a = 0; a < 8; a++)
            CK(cudaMemcpyAsync(dst[a], st + a * n, sizeof(double) * n, cudaMemcpyHostToDevice, m->stream));
    } else {
        unsigned char *st = (unsigned char *)stage(m, sizeof(float) * 8 * n);
        if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
        uint32_t *qx = (uint32_t *)st, *qy = qx + n;
        float *fl = (float *)(qy + n);
        for (long long l = 0; l < n; l++) {
            const double Xw = f->x[l] - m->g.Lx * std::floor(f->x[l] / m->g.Lx);
            const double Yw = f->y[l] - m->g.Ly * std::floor(f->y[l] / m->g.Ly);
            qx[l] = to_fix(Xw / m->g.Lx);
            qy[l] = to_fix(Yw / m->g.Ly);
            fl[l] = (float)f->theta[l];
            fl[n + l] = (float)f->u[l];
            fl[2 * n + l] = (float)f->v[l];
            fl[3 * n + l] = (float)f->omega[l];
            fl[4 * n + l] = (float)f->r[l];
            fl[5 * n + l] = (float)f->h[l];
        }
        DevState32 &s = m->t32[m->tcur];
        CK(cudaMemcpyAsync(s.xq, qx, 4 * n, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(s.yq, qy, 4 * n, cudaMemcpyHostToDevice, m->stream));
        float *dst[6] = {s.th, s.u, s.v, s.w, s.r, s.h};
        for (int a = 0; a < 6; a++)
            CK(cudaMemcpyAsync(dst[a], fl + a * n, 4 * n, cudaMemcpyHostToDevice, m->stream));
    }
    CK(cudaMemsetAsync(m->d_fd, 0, (m->precision == MS_FP64 ? 8 : 4) * 3 * n, m->stream));
    return MS_OK;
}

static Geo32 geo32(double Lx, double Ly, int nx, int ny, double dt)
{
    Geo32 k;
    k.sx = (float)(Lx / 4294967296.0);
    k.sy = (float)(Ly / 4294967296.0);
    k.isx = (float)(4294967296.0 / Lx);
    k.isy = (float)(4294967296.0 / Ly);
    k.inx = (float)(1.0 / nx);
    k.iny = (float)(1.0 / ny);
    k.Lx = (float)Lx;
    k.Ly = (float)Ly;
    k.iLx = (float)(1.0 / Lx);
    k.iLy = (float)(1.0 / Ly);
    k.dt = (float)dt;
    return k;
}

static StepCommon step_common(ms_model *m, long long i_local, double *mom, double *win)
{
    StepCommon sc;
    sc.k = geo32(m->g.Lcx, m->g.Lcy, m->g.nx, m->g.nyr, m->dt);
    sc.nl = m->nl;
    sc.live = nullptr;
    sc.off = m->d_off;
    sc.order = m->d_order;
    sc.order0 = m->d_order;
    sc.skip = nullptr;
    sc.ncell = m->ncell;
    sc.max_n = m->max_n;
    sc.mom = mom;
    sc.win = win;
    sc.tgt = m->d_tgt;
    sc.ctrl = m->d_ctrl;
    sc.g = m->g;
    sc.dt = m->dt;
    sc.N0 = m->fc.N0;
    sc.n_t = m->fc.n_t;
    sc.couple = m->fc.couple;
    sc.i_local = i_local;
    sc.carry_in = m->d_carry;
    sc.carry_out = m->d_carry;
    sc.ncarry = m->n;
    return sc;
}

static CoarseArgs coarse_args(ms_model *m)
{
    CoarseArgs a;
    a.nx = m->g.nx;
    a.ny = m->g.ny;
    a.nyr = m->g.nyr;
    a.nens = m->g.nens;
    a.walls = m->g.walls;
    a.cmax = m->d_cmax;
    a.dx = m->g.Lcx;
    a.dy = m->g.Lcy;
    a.Ac = m->g.Lcx * m->g.Lcy;
    a.dT = (double)m->fc.N0 * m->dt;
    a.N0 = m->fc.N0;
    a.mom = m->d_mom;
    a.win = m->d_win;
    a.q0 = m->d_q0;
    a.q1 = m->d_q1;
    a.V = m->d_V;
    a.S = m->d_S;
    a.tgt = m->d_tgt;
    a.ctrl = m->d_ctrl;
    return a;
}

static bool hybrid_on(const ms_model *m) { return m->hybrid_mode >= 0 && m->fc.couple && m->precision == MS_FP32; }

// drag floor of the closure's relative error: the drag of a 1 cm/s relative
// velocity on 1 m of ice
static double floor_acc(const ms_model *m) { return m->fc.Cd * m->fc.rho_o / m->fc.rho_ice * 1e-4; }

// step facts of fine step i_local of the interval, for the model's state or
// (scratch_out) for the out-of-place timing copies
static StepCommon cell_common(ms_model *m, long long i_local, bool scratch_out)
{
    StepCommon sc = step_common(m, i_local, scratch_out ? m->d_xmom : m->d_mom,
                                scratch_out ? m->d_xwin : m->d_win);
    sc.nl = scratch_out ? m->xnl : m->nl;
    if (scratch_out) sc.carry_out = m->d_xcarry;
    if (hybrid_on(m)) {
        sc.order = m->d_order2;
        sc.live = m->d_live;
        sc.skip = m->d_isc;
    }
    return sc;
}

// the cell kernels of a whole coarse interval (FP32 variants 2 and 3): every
// size class's N0 steps on its own stream, forked once
static cudaError_t launch_interval_cells(ms_model *m, bool scratch_out)
{
    const StepCommon sc = cell_common(m, 0, scratch_out);
    cudaError_t e = cell_fork(m->cl, m->stream);
    if (e == cudaSuccess) e = launch_cell_run32(m->s32, scratch_out ? m->x32 : m->s32, m->P32, sc, m->cl, m->interval);
    if (e == cudaSuccess) e = cell_join(m->cl, m->stream);
    return e;
}

static bool interval_cells(const ms_model *m) { return m->precision == MS_FP32 && m->cl.variant >= 2; }

// cell-kernel launches of one coarse interval on the graph path
static int64_t interval_launches(const ms_model *m)
{
    if (m->cl.variant == 0 || m->precision == MS_FP64) return m->interval;
    int64_t k = 0;
    for (int s = 0; s < m->cl.nseg; s++)
        k += (m->cl.seg_kind[s] >= 2 || (m->cl.variant == 3 && m->cl.seg_kind[s] == 1)) ? 1 : m->interval;
    return k;
}

static cudaError_t launch_step(ms_model *m, long long i_local, bool scratch_out)
{
    StepCommon sc = cell_common(m, i_local, scratch_out);
    if (m->precision == MS_FP64)
        return launch_cell_step64(m->s64, scratch_out ? m->x64 : m->s64, m->P64, sc, m->cl, m->stream);
    return launch_cell_step32(m->s32, scratch_out ? m->x32 : m->s32, m->P32, sc, m->cl, m->stream);
}

// the work that closes a coarse interval: coarse step (coupled) or base += N0
static cudaError_t launch_interval_end(ms_model *m)
{
    if (hybrid_on(m)) {
        // the interval's tendencies (measured or predicted) become the next
        // interval's lagged features; the window is still unconsumed here
        const bool net = m->hybrid_mode == 0 || m->hybrid_mode == 2;
        cudaError_t e = launch_collect_targets(m->d_mom0, m->d_mom, m->d_win, m->ncell, m->fc.N0,
                                               (double)m->fc.N0 * m->dt, m->d_isc, m->d_Yuse, m->d_ctrl, m->d_Ylag,
                                               nullptr, net ? m->d_Yp : nullptr, floor_acc(m),
                                               net ? m->d_nerr : nullptr, net ? m->d_age : nullptr, m->stream);
        if (e != cudaSuccess) return e;
    }
    if (m->fc.couple) return launch_coarse_step(coarse_args(m), m->stream);
    return launch_advance(m->d_ctrl, m->interval, m->stream);
}

// Start of a coarse interval in closure-plus-fallback mode: features, network,
// residual check, the particle cells of each size class, closure cells' update.
static cudaError_t launch_interval_start(ms_model *m)
{
    if (!hybrid_on(m)) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(m->d_mom0, m->d_mom, sizeof(double) * m->ncell * NMOM, cudaMemcpyDeviceToDevice,
                                    m->stream);
    if (e == cudaSuccess)
        e = launch_features(m->d_mom, m->d_tgt, m->ncell, m->g, m->P64, m->d_ctrl, m->dt, m->fc.N0, m->fc.n_t,
                            m->d_Ylag, m->d_ocean, m->d_X, m->stream);
    if (e != cudaSuccess) return e;
    if ((m->hybrid_mode == 0 || m->hybrid_mode == 2) &&
        ms_mlp_forward_device(m->mlp, m->d_X, m->ncell, m->d_Yp, m->stream) != MS_OK)
        return cudaErrorUnknown;
    HybridArgs h{};
    h.X = m->d_X;
    h.Yp = m->d_Yp;
    h.mom = m->d_mom;
    h.mom_rw = m->d_mom;
    h.ncell = m->ncell;
    h.nseg = m->cl.nseg;
    h.P64 = m->P64;
    h.P32 = m->P32;
    h.rho_ice = m->fc.rho_ice;
    h.tol = m->hybrid_tol;
    h.floor_acc = floor_acc(m);
    h.nerr = m->d_nerr;
    h.age = m->d_age;
    h.dT = (double)m->fc.N0 * m->dt;
    h.box = m->d_box;
    h.mode = m->hybrid_mode;
    h.ctrl = m->d_ctrl;
    h.is_closure = m->d_isc;
    h.Yuse = m->d_Yuse;
    h.order = m->d_order;
    h.seg_begin = m->d_segb;
    h.seg_end = m->d_sege;
    h.off = m->d_off;
    h.order2 = m->d_order2;
    h.live = m->d_live;
    h.closure_count = m->d_ccount;
    h.st32 = m->s32;
    h.win = m->d_win;
    h.tgt = m->d_tgt;
    h.N0 = m->fc.N0;
    h.n_t = m->fc.n_t;
    // the resident classes (kind 3) skip closure cells in their own groups;
    // the class of shared blocks keeps a group's closure all or nothing
    h.seg_mask = 0u;
    h.vgroups = nullptr;
    h.vitems = m->cl.ritems;
    h.nvgroups = 0;
    for (int s = 0; s < m->cl.nseg; s++) {
        if (m->cl.seg_kind[s] != 3) h.seg_mask |= 1u << s;
        else if (m->cl.seg_maxn[s] == RUN_T) {
            h.vgroups = m->cl.rgroups[s];
            h.nvgroups = m->cl.rngroups[s];
        }
    }
    return launch_hybrid_select(h, m->stream);
}

static void drop_graph(ms_model *m)
{
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    if (m->gexec_end) cudaGraphExecDestroy(m->gexec_end);
    m->gexec = nullptr;
    m->gexec_end = nullptr;
}

// a sharded model exchanges the coarse inputs before each coarse step
static bool sharded_coarse(const ms_model *m) { return m->shard_nranks > 0 && m->fc.couple; }

// pack this rank's coarse inputs (end of an interval, before the exchange)
static cudaError_t launch_shard_send(ms_model *m)
{
    return launch_shard_pack(m->d_mom, m->d_win, m->ncell, m->d_shard_cells + m->shard_first, m->shard_nown,
                             m->d_send, m->stream);
}

// every rank's coarse inputs into the moments and window sums (after it)
static cudaError_t launch_shard_recv(ms_model *m)
{
    return launch_shard_scatter(m->d_mom, m->d_win, m->ncell, m->d_shard_cells, m->d_shard_rows, m->d_recv,
                                m->stream);
}

template <class F>
static cudaError_t capture(ms_model *m, cudaGraphExec_t *out, F &&body)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = body();
    e = cudaStreamEndCapture(m->stream, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

// One coarse interval as a graph; a sharded model's splits at the exchange
// (gexec ends with the pack of its send rows, gexec_end is the scatter of
// the gathered rows and the coarse step).
static cudaError_t build_graph(ms_model *m)
{
    const bool split = sharded_coarse(m);
    cudaError_t e = capture(m, &m->gexec, [&]() {
        cudaError_t le = launch_interval_start(m);
        // FP32 size classes: one fork per interval, so that a class's next
        // step does not wait for the other classes' current one
        if (le == cudaSuccess && interval_cells(m)) le = launch_interval_cells(m, false);
        else
            for (int i = 0; i < m->interval && le == cudaSuccess; i++) le = launch_step(m, i, false);
        if (le == cudaSuccess) le = split ? launch_shard_send(m) : launch_interval_end(m);
        return le;
    });
    if (e == cudaSuccess && split) e = capture(m, &m->gexec_end, [&]() {
        cudaError_t le = launch_shard_recv(m);
        return le == cudaSuccess ? launch_interval_end(m) : le;
    });
    if (e != cudaSuccess) drop_graph(m);
    return e;
}

// the caller's exchange between the pack and the scatter
static int shard_exchange(ms_model *m)
{
    Trace tr("msdem.shard exchange");
    if (m->exch(m->exch_ctx, (void *)m->stream) != 0) {
        m->exch_failed = true;
        return fail(MS_ERR_ARG, "the exchange of the coarse inputs failed at step %lld", m->steps);
    }
    return MS_OK;
}

static int read_errors(ms_model *m)
{
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (c.err & ERR_TIMEOUT) return fail(MS_ERR_TIMEOUT, "a bounded device wait ran out");
    if (c.err & ERR_NONFINITE) return fail(MS_ERR_UNSTABLE, "floe state became non-finite");
    if (c.err & ERR_CFL)
        return fail(MS_ERR_UNSTABLE, "coarse step needs N1 = %d > %d Lax-Friedrichs substeps", c.N1, NSUB_MAX);
    if (m->mlp && m->hybrid_mode >= 0) return ms_mlp_check(m->mlp);   // the closure network's own waits
    return MS_OK;
}

static void fill_phys(ms_model *m)
{
    const ms_forcing &f = m->fc;
    Phys<double> &P = m->P64;
    Phys<float> &Q = m->P32;
    std::memset(&P, 0, sizeof(P));
    std::memset(&Q, 0, sizeof(Q));
    P.uo_x = f.uo_x; P.uo_y = f.uo_y;
    P.n_modes = Q.n_modes = f.n_modes + f.n_vmodes;
    const double Lcx = m->grid.Lx / m->grid.nx, Lcy = m->grid.Ly / m->grid.ny;
    Q.taylor = 1;
    for (int k = 0; k < P.n_modes; k++) {
        const bool sf = k < f.n_modes;          // stream-function mode (integer wave numbers)
        const double *md = sf ? &m->modes[4 * k] : &m->vmodes[5 * (k - f.n_modes)];
        double kx, ky, ph, Au, Av, Az, Ad;
        if (sf) {
            kx = 2.0 * PI_D * md[1] / m->grid.Lx;
            ky = 2.0 * PI_D * md[2] / m->grid.Ly;
            ph = md[3];
            Au = md[0] * ky;
            Av = md[0] * kx;
            Az = md[0] * (kx * kx + ky * ky);
            Ad = 0.0;
            P.mA[k] = md[0];
            Q.mkx[k] = (int)md[1];
            Q.mky[k] = (int)md[2];
            Q.kdx[k] = (float)md[1];
            Q.kdy[k] = (float)md[2];
        } else {
            kx = md[2];
            ky = md[3];
            ph = md[4];
            Au = -md[0];
            Av = md[1];
            Az = md[1] * kx - md[0] * ky;
            Ad = md[0] * kx + md[1] * ky;
            Q.kdx[k] = (float)(kx * m->grid.Lx / (2.0 * PI_D));
            Q.kdy[k] = (float)(ky * m->grid.Ly / (2.0 * PI_D));
        }
        P.mKx[k] = kx; P.mKy[k] = ky; P.mPh[k] = ph;
        P.mAu[k] = Au; P.mAv[k] = Av; P.mAz[k] = Az; P.mAd[k] = Ad;
        Q.isint[k] = P.isint[k] = sf ? 1 : 0;
        double cyc = ph / (2.0 * PI_D);
        cyc -= std::floor(cyc);
        Q.mCyc[k] = (float)cyc;
        Q.bx[k] = kx * Lcx / (2.0 * PI_D);
        Q.by[k] = ky * Lcy / (2.0 * PI_D);
        Q.bph[k] = cyc;
        Q.kcx[k] = (float)Q.bx[k];
        Q.kcy[k] = (float)Q.by[k];
        Q.mAu[k] = (float)Au;
        Q.mAv[k] = (float)Av;
        Q.mAz[k] = (float)Az;
        Q.mAd[k] = (float)Ad;
        Q.mA[k] = (float)P.mA[k];
        Q.ta[k] = (float)(kx * Lcx);
        Q.tb[k] = (float)(ky * Lcy);
        Q.mKx[k] = (float)kx;      // rad per metre: the gradient of the mode in the ocean expansion
        Q.mKy[k] = (float)ky;
        // small-angle form of the per-floe phase: valid when no mode turns
        // by more than 1/16 cycle across one cell
        if ((std::fabs(kx) * Lcx + std::fabs(ky) * Lcy) / (2.0 * PI_D) > 1.0 / 16.0) Q.taylor = 0;
    }
    // Variant 5 evaluates the current at a floe from its first-order Taylor
    // expansion about a nearby centre.  The neglected term is at most
    // 1/2 |d|^2 sum_m |A_m| |k_m|^2 per component (A_m the mode's velocity or
    // curl amplitude), so |d| <= 2^-11.5 / k_max keeps it below 2^-24 of
    // sum_m |A_m|, i.e. below the FP32 rounding of the mode sum itself.
    {
        double kmax = 0.0;
        for (int k = 0; k < P.n_modes; k++) kmax = std::max(kmax, std::hypot(P.mKx[k], P.mKy[k]));
        const double dmax = kmax > 0.0 ? std::pow(2.0, -11.5) / kmax : 1.0e30;
        Q.ocean_d2 = (float)std::min(dmax * dmax, 1.0e30);
    }
    P.drag_o = f.Cd * f.rho_o * PI_D;
    P.drag_a = f.Ca * f.rho_a * PI_D;
    P.wind_x = f.wind_x; P.wind_y = f.wind_y;
    P.wind_w = f.wind_period > 0.0 ? 2.0 * PI_D / f.wind_period : 0.0;
    P.mass_c = f.rho_ice * PI_D;
    P.inertia_f = f.inertia_half ? 0.5 : 1.0;
    P.E = f.E; P.G = f.G; P.eta = f.eta; P.mu = f.mu; P.inv_h_ref = 1.0 / f.h_ref;
    Q.uo_x = (float)P.uo_x; Q.uo_y = (float)P.uo_y;
    Q.drag_o = (float)P.drag_o; Q.drag_a = (float)P.drag_a;
    Q.wind_x = (float)P.wind_x; Q.wind_y = (float)P.wind_y; Q.wind_w = (float)P.wind_w;
    Q.mass_c = (float)P.mass_c; Q.inertia_f = (float)P.inertia_f;
    Q.E = (float)P.E; Q.G = (float)P.G; Q.eta = (float)P.eta; Q.mu = (float)P.mu;
    Q.inv_h_ref = (float)P.inv_h_ref;
}

// Binned variant: split the cells (largest first) into size classes, each
// launched with a block size and shared memory that fit its largest cell.
static void make_segments(ms_model *m, CellLaunch &c)
{
    const SizeClass *cls = c.variant == 5   ? kClassesV5
                           : c.variant == 4 ? kClassesV4
                                            : (c.variant >= 2 ? kClassesV2 : kClassesV1);
    const int ncls = c.variant == 5   ? (int)(sizeof(kClassesV5) / sizeof(SizeClass))
                     : c.variant == 4 ? (int)(sizeof(kClassesV4) / sizeof(SizeClass))
                     : c.variant >= 2 ? (int)(sizeof(kClassesV2) / sizeof(SizeClass))
                                      : (int)(sizeof(kClassesV1) / sizeof(SizeClass));
    c.nseg = 0;
    c.nbmax = 32;
    int item = 0;
    const int nc = m->ncell;
    auto ncount = [&](int it) { const int cc = m->h_order[it]; return m->h_off[cc + 1] - m->h_off[cc]; };
    for (int s = 0; s < ncls && item < nc; s++) {
        const int lo = (s + 1 < ncls) ? cls[s + 1].hi : -1;
        int e = item;
        while (e < nc && ncount(e) > lo) e++;
        if (e == item) continue;
        c.seg_begin[c.nseg] = item;
        c.seg_end[c.nseg] = e;
        c.seg_kind[c.nseg] = cls[s].kind;
        c.seg_maxn[c.nseg] = cls[s].kind >= 1 ? cls[s].hi : std::max(1, ncount(item));
        c.seg_threads[c.nseg] = cls[s].threads;
        c.nseg++;
        item = e;
    }
    for (int k = 0; k < MAXSEG; k++) {
        c.side[k] = m->side_stream[k];
        c.ev_join[k] = m->ev_join[k];
    }
    c.ev_fork = m->ev_fork;
}

// Variant 5 keeps each floe's window sums since the last gradual update in
// the carry between runs; before the state is replaced or another variant
// takes over inside a coarse interval they go into the window.
static cudaError_t fold_carry(ms_model *m)
{
    if (m->precision != MS_FP32 || m->cl.variant != 5 || !m->fc.couple || m->steps % m->interval == 0)
        return cudaSuccess;
    const StepCommon sc = step_common(m, m->steps % m->interval, m->d_mom, m->d_win);
    return launch_carry_flush(m->s32, sc, m->d_carry, m->n, m->stream);
}

// Variant 5: the cells of the resident classes packed into the groups one
// block takes.  A cell of more than 512 floes opens a group of 4 floes per
// thread (1024 floes), one of more than 256 a group of 2 per thread; smaller
// cells go, largest first, into the open group with the least room that
// still fits them (at most RUN_GCMAX cells), else open a group of one floe
// per thread.  Each class's groups run in decreasing order of floes.  Each
// cell gets about sqrt(n)/beta bins per side, at most sqrt(n) (so a group's
// bins fit its shared memory), none below 3.
static int build_groups(ms_model *m, CellLaunch &cl)
{
    struct G {
        int K, room, nf;
        std::vector<int> cells;
    };
    std::vector<G> gs;
    const int cap_max = 4 * RUN_T;
    std::vector<std::vector<int>> by_room(cap_max + 1);   // open groups by free floes
    auto ncount = [&](int cc) { return m->h_off[cc + 1] - m->h_off[cc]; };
    auto place = [&](int gi, int cc) {
        G &g = gs[gi];
        const int n = ncount(cc);
        g.cells.push_back(cc);
        g.nf += n;
        g.room -= n;
        // only groups of one floe per thread take further cells: a cell's
        // floes then run the code of its own size class wherever it is
        // packed (the 2- and 4-floe classes compile to other instruction
        // sequences, whose rounding may differ)
        if (g.K == 1 && (int)g.cells.size() < RUN_GCMAX) by_room[g.room].push_back(gi);
    };
    int first_item = -1, end_item = -1;
    for (int s = 0; s < cl.nseg; s++)
        if (cl.seg_kind[s] == 3) {
            if (first_item < 0) first_item = cl.seg_begin[s];
            end_item = cl.seg_end[s];
        }
    for (int it = std::max(first_item, 0); it < end_item; it++) {
        const int cc = m->h_order[it], n = ncount(cc);
        if (n > RUN_T) {
            const int K = n > 2 * RUN_T ? 4 : 2;
            gs.push_back(G{K, K * RUN_T, 0, {}});
            place((int)gs.size() - 1, cc);
            continue;
        }
        int found = -1;
        for (int room = n; room <= cap_max && found < 0; room++) {
            auto &b = by_room[room];
            while (!b.empty()) {
                const int gi = b.back();
                b.pop_back();
                if (gs[gi].room == room && (int)gs[gi].cells.size() < RUN_GCMAX) {   // still current
                    found = gi;
                    break;
                }
            }
        }
        if (found < 0) {
            gs.push_back(G{1, std::max(std::min(cl.run_cap1, RUN_T), n), 0, {}});
            found = (int)gs.size() - 1;
        }
        place(found, cc);
    }
    std::vector<int4> groups, items;
    items.reserve(m->ncell);
    for (int s = 0; s < cl.nseg; s++) {
        if (cl.seg_kind[s] != 3) continue;
        const int K = cl.seg_maxn[s] / RUN_T;
        std::vector<int> mine;
        for (int gi = 0; gi < (int)gs.size(); gi++)
            if (gs[gi].K == K) mine.push_back(gi);
        std::stable_sort(mine.begin(), mine.end(), [&](int a, int b) { return gs[a].nf > gs[b].nf; });
        const int first = (int)groups.size();
        for (int gi : mine) {
            int4 g = make_int4((int)items.size(), 0, 0, 0);
            for (int cc : gs[gi].cells) {
                const int n = ncount(cc);
                int nb = (int)std::floor(std::sqrt((double)n) / cl.bin_beta);
                nb = std::min(nb, (int)std::floor(std::sqrt((double)n)));
                if (nb < 3) nb = 0;
                items.push_back(make_int4(cc, g.z, nb, g.w));
                g.y++;
                g.z += n;
                g.w += nb * nb + 1;
            }
            groups.push_back(g);
        }
        cl.rgroups[s] = m->d_rgroups + first;
        cl.rngroups[s] = (int)groups.size() - first;
    }
    cl.ritems = m->d_ritems;
    if ((long long)groups.size() > m->ncell || (long long)items.size() > m->ncell)
        return fail(MS_ERR_STATE, "variant 5 grouping overflow");
    if (!groups.empty())
        CK(cudaMemcpyAsync(m->d_rgroups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice,
                           m->stream));
    if (!items.empty())
        CK(cudaMemcpyAsync(m->d_ritems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                           m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return MS_OK;
}

static int configure_launch(ms_model *m, const CellLaunch &cl_in)
{
    CellLaunch cl = cl_in;
    if (cl.variant == 0 && hybrid_on(m)) return fail(MS_ERR_STATE, "the closure needs a binned cell kernel");
    if (cl.variant == 5 && m->precision != MS_FP32) return fail(MS_ERR_ARG, "variant 5 is FP32 only");
    if (cl.variant != 5 && m->cl.variant == 5) CK(fold_carry(m));
    if (cl.variant >= 1) make_segments(m, cl);
    else cl.nseg = 0;
    if (cl.variant == 5) {
        const int rc = build_groups(m, cl);
        if (rc) return rc;
    }
    // packed warps: consecutive cells of the class, at most 32 floes and 32
    // cells per warp
    cl.pack = m->d_pack;
    cl.npack = 0;
    for (int s = 0; s < cl.nseg; s++) {
        if (cl.seg_kind[s] != 2) continue;
        std::vector<int2> pk;
        int first = cl.seg_begin[s], cnt = 0, sum = 0;
        for (int it = cl.seg_begin[s]; it < cl.seg_end[s]; it++) {
            const int cc = m->h_order[it], nf = m->h_off[cc + 1] - m->h_off[cc];
            if (cnt > 0 && (sum + nf > 32 || cnt == 32)) {
                pk.push_back(make_int2(first, cnt));
                first = it;
                cnt = 0;
                sum = 0;
            }
            cnt++;
            sum += nf;
        }
        if (cnt > 0) pk.push_back(make_int2(first, cnt));
        cl.npack = (int)pk.size();
        CK(cudaMemcpyAsync(m->d_pack, pk.data(), sizeof(int2) * pk.size(), cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    if (m->d_segb && cl.nseg > 0) {
        CK(cudaMemcpyAsync(m->d_segb, cl.seg_begin, sizeof(int) * cl.nseg, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_sege, cl.seg_end, sizeof(int) * cl.nseg, cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    const size_t smem = cell_step_smem(m->precision, cl, m->max_n, m->g.nx, m->g.ny);
    if (smem > 227 * 1024) return fail(MS_ERR_ARG, "cell of %d floes needs %zu B of shared memory", m->max_n, smem);
    CK(cell_step_prepare(m->precision, cl, smem));
    CK(invalidate_lists(m));
    m->cl = cl;
    drop_graph(m);
    return MS_OK;
}

// Grid of bins of side > 2 rad on the domain (fewer than 3 bins along an
// axis: one bin on that axis), at most 2^20 bins.
static void truth_grid(const ms_model *m, double rad, int &nbx, int &nby)
{
    nbx = (int)std::floor(m->g.Lx / (2.0002 * rad));
    nby = (int)std::floor(m->g.Ly / (2.0002 * rad));
    if (nbx < 3) nbx = 1;
    if (nby < 3) nby = 1;
    while ((long long)nbx * nby > (1LL << 20)) {
        if (nbx >= nby) nbx = std::max(3, nbx / 2); else nby = std::max(3, nby / 2);
    }
}

// Bins of the truth DEM.  One grid of bins wider than 2 r_max holds every
// contact partner of a floe in its 3 x 3 neighbourhood; with a wide radius
// distribution most floes are small and such bins hold many candidates, so
// floes of radius <= r_split go to a finer grid and only the larger ones to
// the 2 r_max grid.  r_split is the fraction of r_max (1, 1/2, ..., 1/8) that
// minimises the expected work of a floe's search: candidates tested (bins
// visited times the mean floes per bin, from the actual radii) and bins
// visited.
static int setup_truth_bins(ms_model *m, const double *r, double rmax)
{
    const long long n = m->n;
    int nbx, nby, nbx2, nby2;
    truth_grid(m, rmax, nbx2, nby2);
    double best = -1.0, best_q = 1.0;
    for (double q : {1.0, 0.5, 1.0 / 3.0, 0.25, 1.0 / 6.0, 0.125}) {
        const double rs = q * rmax;
        truth_grid(m, rs, nbx, nby);
        long long nS = 0;
        for (long long l = 0; l < n; l++) nS += r[l] <= rs ? 1 : 0;
        const long long nL = n - nS;
        const double dS = (double)nS / ((double)nbx * nby), dL = nL ? (double)nL / ((double)nbx2 * nby2) : 0.0;
        const double Bx = m->g.Lx / nbx, By = m->g.Ly / nby;
        const double large_bins = std::min(3, nbx2) * (double)std::min(3, nby2);
        // a visited bin costs about half a candidate test (its bounds, the loop)
        double cost = 0.0;
        for (long long l = 0; l < n; l++) {
            const int kx = (int)std::ceil((r[l] + rs) / Bx), ky = (int)std::ceil((r[l] + rs) / By);
            const double bins = std::min(2 * kx + 1, nbx) * (double)std::min(2 * ky + 1, nby);
            cost += bins * (dS + 0.5) + (nL ? large_bins * (dL + 0.5) : 0.0);
        }
        if (best < 0.0 || cost < 0.9 * best) {   // a finer grid only for a clear gain
            best = cost;
            best_q = q;
        }
    }
    truth_grid(m, best_q * rmax, nbx, nby);
    long long nL = 0;
    for (long long l = 0; l < n; l++) nL += r[l] <= best_q * rmax ? 0 : 1;
    TruthBins *bs[2] = {&m->tb, &m->cb};
    const int dims[2][4] = {{nbx, nby, nL ? nbx2 : 0, nL ? nby2 : 0}, {m->g.nx, m->g.ny, 0, 0}};
    for (int k = 0; k < 2; k++) {
        TruthBins &b = *bs[k];
        b.nbx = dims[k][0];
        b.nby = dims[k][1];
        b.nbx2 = dims[k][2];
        b.nby2 = dims[k][3];
        b.r_split = k == 0 ? (float)(best_q * rmax) : 0.0f;
        const int nbins = b.nbins();
        b.nscan_blocks = (nbins + 1023) / 1024;
        if (b.nscan_blocks > 1024) return fail(MS_ERR_ARG, "too many bins (%d)", nbins);
        CK(dalloc(m, &b.count, nbins));
        CK(dalloc(m, &b.start, nbins + 1));
        CK(dalloc(m, &b.cursor, nbins));
        CK(dalloc(m, &b.sorted, m->n));
        CK(dalloc(m, &b.bin, m->n));
        CK(dalloc(m, &b.scan_tmp, b.nscan_blocks));
        const int nn = (int)m->n;
        CK(cudaMemcpyAsync(b.start + nbins, &nn, sizeof(int), cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    return MS_OK;
}

// ================================================================== C-ABI
extern "C" {

const char *ms_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------- checkpoint
// File layout: an 8-byte tag, then (for every item below, in this order) an
// int64 byte count, the bytes, and the 64-bit FNV-1a hash of those bytes.
// ms_load reads and checks the whole file before it changes the model, so a
// truncated or corrupted file (a flipped byte in a candidate list would
// otherwise index past its cell) is refused with the model left as it was.
// Items: the header (precision,
// sizes, schedule counters, dt, launch choice), the cell offsets (the layout
// the state is stored in), the msDEM state in cell order, the per-cell
// moments, window sums, coarse state and gradual-update targets, the device
// control block, the candidate lists and the running window sums (FP32),
// and the truth DEM's current state with its last drag.
namespace {
constexpr char CK_TAG[8] = {'M', 'S', 'D', 'E', 'M', 'C', 'K', '2'};

// 64-bit FNV-1a (Fowler, Noll, Vo) of a byte string
uint64_t fnv1a64(const void *p, size_t bytes)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < bytes; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct CkHeader {
    int32_t precision, nens, walls, variant, threads, persistent;
    int64_t n, ncell, steps, truth_steps;
    double dt, truth_dt, bin_beta;
};

struct CkItem {
    void *dev;      // device pointer, or nullptr for a host item
    void *host;
    size_t bytes;
};
}  // namespace

// the device arrays of a model's state, in file order
static std::vector<CkItem> ck_items(ms_model *m)
{
    std::vector<CkItem> it;
    const size_t n = (size_t)m->n, nc = (size_t)m->ncell;
    auto dev = [&](void *p, size_t bytes) { it.push_back({p, nullptr, bytes}); };
    if (m->precision == MS_FP64) {
        double *a[8] = {m->s64.x, m->s64.y, m->s64.th, m->s64.u, m->s64.v, m->s64.w, m->s64.r, m->s64.h};
        for (double *p : a) dev(p, 8 * n);
    } else {
        dev(m->s32.xq, 4 * n);
        dev(m->s32.yq, 4 * n);
        float *a[6] = {m->s32.th, m->s32.u, m->s32.v, m->s32.w, m->s32.r, m->s32.h};
        for (float *p : a) dev(p, 4 * n);
    }
    dev(m->d_mom, sizeof(double) * NMOM * nc);
    dev(m->d_win, sizeof(double) * NWIN * nc);
    dev(m->d_q0, sizeof(double) * 4 * nc);
    dev(m->d_tgt, sizeof(double) * 4 * nc);
    dev(m->d_ctrl, sizeof(Ctrl));
    if (m->precision == MS_FP32 && m->nl.head) {
        dev(m->nl.head, sizeof(uint4) * n);
        dev(m->nl.tail, sizeof(uint4) * NLT * n);
        dev(m->nl.xb, sizeof(uint2) * n);
        dev(m->nl.cstep, sizeof(long long) * nc);
        dev(m->nl.skin, sizeof(float) * nc);
    }
    if (m->precision == MS_FP32 && m->d_carry) dev(m->d_carry, sizeof(float) * RUN_NCARRY * n);
    if (m->g.nens == 1 && m->n > 0) {
        const size_t es = m->precision == MS_FP64 ? 8 : 4;
        if (m->precision == MS_FP64) {
            const DevState64 &t = m->t64[m->tcur];
            double *a[8] = {t.x, t.y, t.th, t.u, t.v, t.w, t.r, t.h};
            for (double *p : a) dev(p, 8 * n);
        } else {
            const DevState32 &t = m->t32[m->tcur];
            dev(t.xq, 4 * n);
            dev(t.yq, 4 * n);
            float *a[6] = {t.th, t.u, t.v, t.w, t.r, t.h};
            for (float *p : a) dev(p, 4 * n);
        }
        dev(m->d_fd, es * 3 * n);
    }
    return it;
}

int ms_save(ms_model *m, const char *path)
{
    if (!m || !path) return fail(MS_ERR_ARG, "NULL argument");
    Trace tr("msdem.save");
    if (hybrid_on(m)) return fail(MS_ERR_STATE, "detach the closure before a checkpoint");
    CK(cudaStreamSynchronize(m->stream));
    CkHeader h{};
    h.precision = m->precision;
    h.nens = m->g.nens;
    h.walls = m->g.walls;
    h.variant = m->cl.variant;
    h.threads = m->cl.threads;
    h.persistent = m->cl.persistent;
    h.n = m->n;
    h.ncell = m->ncell;
    h.steps = m->steps;
    h.truth_steps = m->truth_steps;
    h.dt = m->dt;
    h.truth_dt = m->truth_dt;
    h.bin_beta = m->cl.bin_beta;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MS_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(CK_TAG, 1, 8, f) == 8;
    auto put = [&](const void *p, size_t bytes) {
        const int64_t b = (int64_t)bytes;
        const uint64_t hash = fnv1a64(p, bytes);
        ok = ok && std::fwrite(&b, sizeof(b), 1, f) == 1 && (bytes == 0 || std::fwrite(p, 1, bytes, f) == bytes) &&
             std::fwrite(&hash, sizeof(hash), 1, f) == 1;
    };
    put(&h, sizeof(h));
    put(m->h_off.data(), sizeof(int) * m->h_off.size());
    std::vector<unsigned char> buf;
    for (const CkItem &it : ck_items(m)) {
        buf.resize(it.bytes);
        if (it.bytes && cudaMemcpy(buf.data(), it.dev, it.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return fail(MS_ERR_CUDA, "reading the state for the checkpoint failed");
        }
        put(buf.data(), it.bytes);
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MS_OK : fail(MS_ERR_ARG, "writing %s failed", path);
}

int ms_load(ms_model *m, const char *path)
{
    if (!m || !path) return fail(MS_ERR_ARG, "NULL argument");
    Trace tr("msdem.load");
    if (hybrid_on(m)) return fail(MS_ERR_STATE, "detach the closure before loading a checkpoint");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MS_ERR_ARG, "cannot open %s", path);
    char tag[8];
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, CK_TAG, 8) == 0;
    bool hash_ok = true;
    auto get = [&](void *p, size_t bytes) {
        int64_t b = -1;
        uint64_t hash = 0;
        ok = ok && std::fread(&b, sizeof(b), 1, f) == 1 && b == (int64_t)bytes &&
             (bytes == 0 || std::fread(p, 1, bytes, f) == bytes) && std::fread(&hash, sizeof(hash), 1, f) == 1;
        if (ok && hash != fnv1a64(p, bytes)) hash_ok = ok = false;
    };
    CkHeader h{};
    get(&h, sizeof(h));
    if (!ok) {
        std::fclose(f);
        return fail(MS_ERR_ARG, "%s is not a checkpoint of this library%s", path, hash_ok ? "" : " (checksum)");
    }
    if (h.precision != m->precision || h.nens != m->g.nens || h.walls != m->g.walls || h.n != m->n ||
        h.ncell != m->ncell) {
        std::fclose(f);
        return fail(MS_ERR_ARG, "checkpoint of another model (precision, floes, cells or boundary differ)");
    }
    std::vector<int> off(m->h_off.size());
    get(off.data(), sizeof(int) * off.size());
    if (!ok || off != m->h_off) {
        std::fclose(f);
        return fail(MS_ERR_ARG, "checkpoint of another floe layout (the floes per cell differ)%s",
                    hash_ok ? "" : " or corrupted (checksum)");
    }
    // every item read and its hash checked before the model changes (the
    // truth state goes into the first of its two copies)
    const int tcur_keep = m->tcur;
    m->tcur = 0;
    const std::vector<CkItem> items = ck_items(m);
    m->tcur = tcur_keep;
    std::vector<std::vector<unsigned char>> bufs(items.size());
    for (size_t i = 0; i < items.size() && ok; i++) {
        bufs[i].resize(items[i].bytes);
        get(bufs[i].data(), items[i].bytes);
    }
    if (ok) {   // nothing may follow the last item
        unsigned char extra;
        ok = std::fread(&extra, 1, 1, f) == 0;
    }
    std::fclose(f);
    if (!ok)
        return fail(MS_ERR_ARG, "%s is %s", path,
                    hash_ok ? "truncated or of another model" : "corrupted (an item's checksum does not match)");
    // the saved launch (configuring a launch forgets the candidate lists;
    // the checkpoint's lists are restored below)
    CellLaunch c = m->cl;
    c.variant = h.variant;
    c.threads = h.threads;
    c.persistent = h.persistent;
    c.bin_beta = (float)h.bin_beta;
    int rc = configure_launch(m, c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(m->stream));
    m->tcur = 0;   // the truth state goes into the first copy
    for (size_t i = 0; i < items.size(); i++) {
        if (items[i].bytes &&
            cudaMemcpy(items[i].dev, bufs[i].data(), items[i].bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(MS_ERR_CUDA, "writing the checkpoint's state to the device failed");
    }
    m->steps = h.steps;
    m->truth_steps = h.truth_steps;
    m->dt = h.dt;
    m->truth_dt = h.truth_dt;
    drop_graph(m);
    return MS_OK;
}

int ms_probe_fp32(int32_t reps, double *tflops)
{
    if (reps < 1 || !tflops) return fail(MS_ERR_ARG, "probe needs reps >= 1 and an output");
    const cudaError_t e = fma_probe(reps, tflops);
    if (e != cudaSuccess) return fail(MS_ERR_CUDA, "FP32 probe: %s", cudaGetErrorString(e));
    return MS_OK;
}

void ms_free(ms_model *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    drop_graph(m);
    for (void *p : m->allocs) cudaFree(p);
    if (m->h_stage) cudaFreeHost(m->h_stage);
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    for (int k = 0; k < MAXSEG; k++) {
        if (m->side_stream[k]) cudaStreamDestroy(m->side_stream[k]);
        if (m->ev_join[k]) cudaEventDestroy(m->ev_join[k]);
    }
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    delete m;
}

int ms_init(ms_model **out, const ms_grid *grid, const ms_floes *floes, const ms_forcing *forcing)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !forcing) return fail(MS_ERR_ARG, "grid or forcing is NULL");
    if (grid->nx < 1 || grid->ny < 1) return fail(MS_ERR_ARG, "grid needs nx, ny >= 1");
    if (grid->nens < 0 || grid->nens > 65536) return fail(MS_ERR_ARG, "nens must be in [0, 65536]");
    if (grid->walls < 0 || grid->walls > 2) return fail(MS_ERR_ARG, "walls must be 0, 1 or 2");
    const int nens = grid->nens > 1 ? grid->nens : 1;
    if ((long long)grid->nx * grid->ny * nens > (1LL << 24)) return fail(MS_ERR_ARG, "more than 2^24 cells");
    if (!(grid->Lx > 0.0) || !(grid->Ly > 0.0) || !isfin(grid->Lx) || !isfin(grid->Ly))
        return fail(MS_ERR_ARG, "domain sides must be positive and finite");
    const ms_forcing &f = *forcing;
    if (f.precision != MS_FP32 && f.precision != MS_FP64) return fail(MS_ERR_ARG, "precision must be MS_FP32 or MS_FP64");
    if (f.n_modes < 0 || f.n_modes > MS_MAX_MODES) return fail(MS_ERR_ARG, "n_modes must be in [0, %d]", MS_MAX_MODES);
    if (f.n_modes > 0 && !f.modes) return fail(MS_ERR_ARG, "modes is NULL");
    for (int k = 0; k < f.n_modes; k++) {
        for (int a = 0; a < 4; a++)
            if (!isfin(f.modes[4 * k + a])) return fail(MS_ERR_ARG, "mode %d is not finite", k);
        if (f.modes[4 * k + 1] != std::floor(f.modes[4 * k + 1]) || f.modes[4 * k + 2] != std::floor(f.modes[4 * k + 2]) ||
            std::fabs(f.modes[4 * k + 1]) > 1024 || std::fabs(f.modes[4 * k + 2]) > 1024)
            return fail(MS_ERR_ARG, "mode %d: wave numbers must be integers of magnitude <= 1024", k);
    }
    if (f.n_vmodes < 0 || f.n_modes + f.n_vmodes > MS_MAX_MODES)
        return fail(MS_ERR_ARG, "n_modes + n_vmodes must be in [0, %d]", MS_MAX_MODES);
    if (f.n_vmodes > 0 && !f.vmodes) return fail(MS_ERR_ARG, "vmodes is NULL");
    for (int k = 0; k < 5 * f.n_vmodes; k++)
        if (!isfin(f.vmodes[k])) return fail(MS_ERR_ARG, "velocity mode %d is not finite", k / 5);
    const double vals[] = {f.uo_x, f.uo_y, f.rho_o, f.Cd, f.rho_a, f.Ca, f.wind_x, f.wind_y, f.wind_period,
                           f.rho_ice, f.E, f.G, f.eta, f.mu, f.h_ref};
    for (double v : vals)
        if (!isfin(v)) return fail(MS_ERR_ARG, "a forcing constant is not finite");
    if (!(f.rho_ice > 0.0) || !(f.h_ref > 0.0)) return fail(MS_ERR_ARG, "rho_ice and h_ref must be positive");
    if (f.E < 0 || f.G < 0 || f.eta < 0 || f.mu < 0 || f.Cd < 0 || f.Ca < 0 || f.rho_o < 0 || f.rho_a < 0 ||
        f.wind_period < 0)
        return fail(MS_ERR_ARG, "material and drag constants must be non-negative");
    if (f.couple && (f.N0 <= 0 || f.n_t <= 0 || f.N0 % f.n_t != 0))
        return fail(MS_ERR_ARG, "coupling needs N0 > 0, n_t > 0 and N0 %% n_t == 0");
    int rc = validate_floes(floes, -1);
    if (rc) return rc;
    if (grid->walls)
        for (long long l = 0; l < floes->n; l++)
            if (!(floes->x[l] >= 0.0 && floes->x[l] < grid->Lx))
                return fail(MS_ERR_ARG, "floe %lld starts outside [0, Lx) between the walls", l);

    ms_model *m = new ms_model();
    m->precision = f.precision;
    m->grid = *grid;
    m->fc = f;
    m->modes.assign(f.modes ? f.modes : nullptr, f.modes ? f.modes + 4 * f.n_modes : nullptr);
    m->fc.modes = m->modes.data();
    m->vmodes.assign(f.vmodes ? f.vmodes : nullptr, f.vmodes ? f.vmodes + 5 * f.n_vmodes : nullptr);
    m->fc.vmodes = m->vmodes.data();
    m->n = floes->n;
    m->ncell = grid->nx * grid->ny * nens;
    m->g = grid_geom(grid);
    m->interval = f.couple ? f.N0 : 100;
    fill_phys(m);

    // reject ambiguous minimum images
    const long long n = m->n;
    double rmax = 0.0;
    for (long long l = 0; l < n; l++) rmax = std::max(rmax, floes->r[l]);
    if (n > 0 && !(2.0 * rmax < 0.5 * std::min(m->g.Lcx, m->g.Lcy))) {
        ms_free(m);
        return fail(MS_ERR_ARG, "2 r_max = %g m must be below half the cell side (%g m)", 2.0 * rmax,
                    0.5 * std::min(m->g.Lcx, m->g.Lcy));
    }

    int dev = 0;
    cudaError_t e;
#define CKM(call)                                                                                 \
    do {                                                                                          \
        if ((e = (call)) != cudaSuccess) {                                                        \
            ms_free(m);                                                                           \
            return fail(MS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e));              \
        }                                                                                         \
    } while (0)
    CKM(cudaGetDevice(&dev));
    CKM(cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev));
    CKM(cudaStreamCreateWithFlags(&m->own_stream, cudaStreamNonBlocking));
    int p_least = 0, p_great = 0;
    CKM(cudaDeviceGetStreamPriorityRange(&p_least, &p_great));
    for (int k = 0; k < MAXSEG; k++) {
        const int pr = k < kHighPriorityClasses ? p_great : p_least;
        CKM(cudaStreamCreateWithPriority(&m->side_stream[k], cudaStreamNonBlocking, pr));
        CKM(cudaEventCreateWithFlags(&m->ev_join[k], cudaEventDisableTiming));
    }
    CKM(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
    m->stream = m->own_stream;
    const int nc = m->ncell;
    CKM(dalloc(m, &m->d_off, nc + 1));
    CKM(dalloc(m, &m->d_order, nc));
    CKM(dalloc(m, &m->d_mom, (size_t)nc * NMOM));
    CKM(dalloc(m, &m->d_win, (size_t)nc * NWIN));
    CKM(dalloc(m, &m->d_xmom, (size_t)nc * NMOM));
    CKM(dalloc(m, &m->d_xwin, (size_t)nc * NWIN));
    CKM(dalloc(m, &m->d_q0, (size_t)nc * 4));
    CKM(dalloc(m, &m->d_q1, (size_t)nc * 4));
    CKM(dalloc(m, &m->d_V, (size_t)nc * 2));
    CKM(dalloc(m, &m->d_S, (size_t)nc * 4));
    CKM(dalloc(m, &m->d_tgt, (size_t)nc * 4));
    CKM(dalloc(m, &m->d_tmom, (size_t)nc * NMOM));
    CKM(dalloc(m, &m->d_ctrl, 1));
    CKM(dalloc(m, &m->d_cmax, nens));
    CKM(dalloc(m, &m->d_pack, nc));
    CKM(dalloc(m, &m->d_raw, 8 * (size_t)n));
    CKM(dalloc(m, &m->d_orig, (size_t)n));
    CKM(dalloc(m, &m->d_cell_of, (size_t)n));
    CKM(dalloc(m, &m->d_first, 2));
    CKM(cudaMemsetAsync(m->d_cmax, 0, sizeof(unsigned long long) * nens, m->stream));
    if (m->precision == MS_FP64) {
        CKM(alloc64(m, m->s64, n));
        if (nens == 1) {
            CKM(alloc64(m, m->t64[0], n));
            CKM(alloc64(m, m->t64[1], n));
        }
        CKM(dalloc(m, (double **)&m->d_fd, 3 * (size_t)n));
    } else {
        CKM(alloc32(m, m->s32, n));
        CKM(alloc_lists(m, m->nl, n, nc));
        CKM(dalloc(m, &m->d_rgroups, nc));
        CKM(dalloc(m, &m->d_ritems, nc));
        CKM(dalloc(m, &m->d_carry, (size_t)RUN_NCARRY * n));
        CKM(dalloc(m, &m->d_xcarry, (size_t)RUN_NCARRY * n));
        CKM(cudaMemsetAsync(m->d_carry, 0, sizeof(float) * RUN_NCARRY * (size_t)n, m->stream));
        if (nens == 1) {
            CKM(alloc32(m, m->t32[0], n));
            CKM(alloc32(m, m->t32[1], n));
        }
        CKM(dalloc(m, (float **)&m->d_fd, 3 * (size_t)n));
    }
    CKM(cudaMemsetAsync(m->d_ctrl, 0, sizeof(Ctrl), m->stream));
    CKM(cudaMemsetAsync(m->d_win, 0, sizeof(double) * nc * NWIN, m->stream));
    CKM(cudaMemsetAsync(m->d_q0, 0, sizeof(double) * nc * 4, m->stream));
    CKM(cudaMemsetAsync(m->d_tgt, 0, sizeof(double) * nc * 4, m->stream));
    // The cell of every floe, the cells' offsets and each cell's floes in the
    // caller's order: a counting sort on the device over the raw upload
    // (cell of each floe and counts, scan, scatter, rank sort within cells).
    // The host keeps the offsets for the launch layout and the permutation
    // for downloads.
    if (n > 0 && (rc = send_raw(m, floes))) {
        ms_free(m);
        return rc;
    }
    {
        int *count = nullptr, *cursor = nullptr, *tmp = nullptr;
        const long long ntmp = sort_scan_ints(nc + 1);
        auto release = [&]() {
            cudaFree(count);
            cudaFree(cursor);
            cudaFree(tmp);
        };
        e = cudaMalloc(&count, sizeof(int) * nc);
        if (e == cudaSuccess) e = cudaMalloc(&cursor, sizeof(int) * nc);
        if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int) * ntmp);
        if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * nc, m->stream);
        if (e == cudaSuccess) e = launch_cell_of(m->d_raw, up_geom(m), m->d_cell_of, count, m->stream);
        if (e == cudaSuccess) e = sort_by_cell(m->d_cell_of, count, m->d_off, cursor, m->d_orig, tmp, nc, n, m->stream);
        m->h_off.assign(nc + 1, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m->h_off.data(), m->d_off, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, m->stream);
        std::vector<int> orig32(n);
        m->h_cell_of_orig.resize(n);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(orig32.data(), m->d_orig, sizeof(int) * n, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(m->h_cell_of_orig.data(), m->d_cell_of, sizeof(int) * n, cudaMemcpyDeviceToHost,
                                m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        release();
        if (e != cudaSuccess) {
            ms_free(m);
            return fail(MS_ERR_CUDA, "cell assignment failed: %s", cudaGetErrorString(e));
        }
        m->h_orig.assign(orig32.begin(), orig32.end());
    }
    for (int c = 0; c < nc; c++) m->max_n = std::max(m->max_n, m->h_off[c + 1] - m->h_off[c]);
    const int cap = m->precision == MS_FP64 ? 2048 : 4096;
    if (m->max_n > cap) {
        const int mx = m->max_n;
        ms_free(m);
        return fail(MS_ERR_ARG, "a cell holds %d floes; at most %d are supported", mx, cap);
    }
    m->h_order.resize(nc);
    for (int c = 0; c < nc; c++) m->h_order[c] = c;
    std::stable_sort(m->h_order.begin(), m->h_order.end(), [&](int a, int b) {
        return (m->h_off[a + 1] - m->h_off[a]) > (m->h_off[b + 1] - m->h_off[b]);
    });
    CKM(cudaMemcpyAsync(m->d_order, m->h_order.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, m->stream));
#undef CKM
    // an ensemble has no truth DEM (each realization's truth is a model of its own)
    if ((rc = raw_to_state(m)) ||
        (nens == 1 && ((rc = upload_truth_state(m, floes)) || (rc = setup_truth_bins(m, floes->r, rmax > 0 ? rmax : 1.0))))) {
        ms_free(m);
        return rc;
    }
    CellLaunch cl{};
    cl.variant = m->precision == MS_FP32 ? 5 : 0;
    cl.threads = 128;
    cl.bin_beta = 1.3f;
    cl.run_skin = 32.0f;
    cl.run_cap1 = RUN_T;
    cl.persistent = 0;
    cl.grid = m->sm_count * 4;
    if (cl.variant >= 1 && configure_launch(m, cl) != MS_OK) cl.variant = 0;   // cells too large to bin in shared memory
    if ((rc = configure_launch(m, cl))) {
        ms_free(m);
        return rc;
    }
    StepCommon sc = step_common(m, 0, m->d_mom, m->d_win);
    e = m->precision == MS_FP64 ? launch_cell_moments64(m->s64, m->P64, sc, m->stream)
                                : launch_cell_moments32(m->s32, m->P32, sc, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        ms_free(m);
        return fail(MS_ERR_CUDA, "initial moments failed: %s", cudaGetErrorString(e));
    }
    *out = m;
    return MS_OK;
}

int ms_set_stream(ms_model *m, void *stream)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    CK(cudaStreamSynchronize(m->stream));
    m->stream = stream ? (cudaStream_t)stream : m->own_stream;
    return MS_OK;
}

static int step_enqueue(ms_model *m, double dt, int64_t nsteps);

int ms_step(ms_model *m, double dt, int64_t nsteps)
{
    int rc = step_enqueue(m, dt, nsteps);
    if (rc) return rc;
    return read_errors(m);
}

int ms_step_async(ms_model *m, double dt, int64_t nsteps) { return step_enqueue(m, dt, nsteps); }

int ms_sync(ms_model *m)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    return read_errors(m);
}

static int step_enqueue(ms_model *m, double dt, int64_t nsteps)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    Trace tr("msdem.step");
    if (!(dt > 0.0) || !isfin(dt)) return fail(MS_ERR_ARG, "dt must be positive and finite");
    if (nsteps < 0) return fail(MS_ERR_ARG, "nsteps < 0");
    if (m->dt == 0.0) m->dt = dt;
    else if (dt != m->dt) return fail(MS_ERR_ARG, "dt = %g differs from the model's dt = %g", dt, m->dt);
    if (m->exch_failed) return fail(MS_ERR_STATE, "an exchange of the coarse inputs failed; the model cannot step");
    const int N = m->interval;
    const bool split = sharded_coarse(m);
    while (nsteps > 0) {
        const long long i_local = m->steps % N;
        if (i_local == 0 && nsteps >= N && !m->graph_failed) {
            if (!m->gexec) {
                cudaError_t e = build_graph(m);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    m->graph_failed = true;
                    drop_graph(m);
                    continue;
                }
            }
            {
                Trace ti("msdem.interval (graph)");
                CK(cudaGraphLaunch(m->gexec, m->stream));
            }
            m->steps += N;
            nsteps -= N;
            if (split) {
                int rc = shard_exchange(m);
                if (rc) return rc;
                CK(cudaGraphLaunch(m->gexec_end, m->stream));
            }
            m->replays++;
            continue;
        }
        if (i_local == 0) {
            Trace ts("msdem.interval start");
            CK(launch_interval_start(m));
        }
        {
            Trace tf("msdem.fine step");
            CK(launch_step(m, i_local, false));
        }
        m->steps++;
        nsteps--;
        if (m->steps % N == 0) {
            Trace te("msdem.interval end (coarse step)");
            if (split) {
                CK(launch_shard_send(m));
                int rc = shard_exchange(m);
                if (rc) return rc;
                CK(launch_shard_recv(m));
            }
            CK(launch_interval_end(m));
        }
    }
    return MS_OK;
}

int ms_moments(ms_model *m, double *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    double *st = (double *)stage(m, sizeof(double) * m->ncell * NMOM);
    if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
    CK(cudaMemcpyAsync(st, m->d_mom, sizeof(double) * m->ncell * NMOM, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    std::memcpy(out, st, sizeof(double) * m->ncell * NMOM);
    return MS_OK;
}

int ms_coupling(ms_model *m, double *q, double *targets, double *window, int64_t *flags)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    const size_t nc = m->ncell;
    if (q) CK(cudaMemcpyAsync(q, m->d_q0, sizeof(double) * 4 * nc, cudaMemcpyDeviceToHost, m->stream));
    if (targets) CK(cudaMemcpyAsync(targets, m->d_tgt, sizeof(double) * 4 * nc, cudaMemcpyDeviceToHost, m->stream));
    if (window) CK(cudaMemcpyAsync(window, m->d_win, sizeof(double) * NWIN * nc, cudaMemcpyDeviceToHost, m->stream));
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (flags) {
        flags[0] = c.have_q;
        flags[1] = c.have_tgt;
        flags[2] = m->steps;
    }
    return MS_OK;
}

static int download(ms_model *m, bool truth, double *out)
{
    Trace tr("msdem.get_floes");
    const long long n = m->n;
    if (n == 0) return MS_OK;
    const int nx = m->g.nx;
    if (m->precision == MS_FP64) {
        double *st = (double *)stage(m, sizeof(double) * 8 * n);
        if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
        const DevState64 &s = truth ? m->t64[m->tcur] : m->s64;
        const double *src[8] = {s.x, s.y, s.th, s.u, s.v, s.w, s.r, s.h};
        for (int a = 0; a < 8; a++)
            CK(cudaMemcpyAsync(st + a * n, src[a], sizeof(double) * n, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));
        host_parallel(n, [&](long long k0, long long k1) {
            for (long long k = k0; k < k1; k++) {
                const long long l = truth ? k : m->h_orig[k];
                const int c = truth ? 0 : m->h_cell_of_orig[l];
                const double X0 = truth ? 0.0 : (c % nx) * m->g.Lcx, Y0 = truth ? 0.0 : (c / nx) * m->g.Lcy;
                out[l] = X0 + st[k];
                out[n + l] = Y0 + st[n + k];
                for (int a = 2; a < 8; a++) out[a * n + l] = st[a * n + k];
            }
        });
    } else {
        unsigned char *st = (unsigned char *)stage(m, sizeof(float) * 8 * n);
        if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
        uint32_t *qx = (uint32_t *)st, *qy = qx + n;
        float *fl = (float *)(qy + n);
        const DevState32 &s = truth ? m->t32[m->tcur] : m->s32;
        CK(cudaMemcpyAsync(qx, s.xq, 4 * n, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaMemcpyAsync(qy, s.yq, 4 * n, cudaMemcpyDeviceToHost, m->stream));
        const float *src[6] = {s.th, s.u, s.v, s.w, s.r, s.h};
        for (int a = 0; a < 6; a++)
            CK(cudaMemcpyAsync(fl + a * n, src[a], 4 * n, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));
        host_parallel(n, [&](long long k0, long long k1) {
            for (long long k = k0; k < k1; k++) {
                const long long l = truth ? k : m->h_orig[k];
                if (truth) {
                    out[l] = from_fix(qx[k]) * m->g.Lx;
                    out[n + l] = from_fix(qy[k]) * m->g.Ly;
                } else {
                    const int c = m->h_cell_of_orig[l];
                    out[l] = ((c % nx) + from_fix(qx[k])) * m->g.Lcx;
                    out[n + l] = ((c / nx) + from_fix(qy[k])) * m->g.Lcy;
                }
                for (int a = 0; a < 6; a++) out[(a + 2) * n + l] = fl[a * n + k];
            }
        });
    }
    return MS_OK;
}

int ms_get_floes(ms_model *m, double *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    return download(m, false, out);
}

static int no_truth(const ms_model *m)
{
    return m->g.nens > 1 ? fail(MS_ERR_STATE, "an ensemble model has no truth DEM") : MS_OK;
}

int ms_truth_get_floes(ms_model *m, double *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    if (no_truth(m)) return MS_ERR_STATE;
    return download(m, true, out);
}

int ms_set_floes(ms_model *m, const ms_floes *floes)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    Trace tr("msdem.set_floes");
    int rc = check_floe_args(floes, m->n);
    if (rc) return rc;
    if (m->n > 0) {
        // checks on the device over the raw copy; the state changes only
        // after both pass
        if ((rc = send_raw(m, floes))) return rc;
        unsigned long long first[2];
        CK(cudaMemsetAsync(m->d_first, 0xff, sizeof(first), m->stream));
        CK(launch_check_floes(m->d_raw, m->d_cell_of, up_geom(m), m->d_first, m->stream));
        CK(cudaMemcpyAsync(first, m->d_first, sizeof(first), cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));
        if (first[0] < (unsigned long long)m->n) {
            const long long l = (long long)first[0];
            if (!floe_finite(floes, l)) return fail(MS_ERR_ARG, "floe %lld has a non-finite value", l);
            return fail(MS_ERR_ARG, "floe %lld has r <= 0 or h <= 0", l);
        }
        if (first[1] < (unsigned long long)m->n) return fail(MS_ERR_ARG, "floe %lld left its cell", (long long)first[1]);
        CK(fold_carry(m));
        if ((rc = raw_to_state(m))) return rc;
    }
    CK(invalidate_lists(m));
    StepCommon sc = step_common(m, 0, m->d_mom, m->d_win);
    CK(m->precision == MS_FP64 ? launch_cell_moments64(m->s64, m->P64, sc, m->stream)
                               : launch_cell_moments32(m->s32, m->P32, sc, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return MS_OK;
}

static cudaError_t truth_one(ms_model *m, int cur, int nxt, long long step)
{
    TruthArgs a;
    a.n = m->n;
    a.g = m->g;
    a.k = geo32(m->g.Lx, m->g.Ly, 1, 1, m->truth_dt);
    a.dt = m->truth_dt;
    a.step = step;
    a.ctrl = m->d_ctrl;
    a.fd = m->d_fd;
    if (m->precision == MS_FP64) return launch_truth_step64(m->t64[cur], m->t64[nxt], m->P64, a, m->tb, m->stream);
    return launch_truth_step32(m->t32[cur], m->t32[nxt], m->P32, a, m->tb, m->stream);
}

int ms_truth_step(ms_model *m, double dt, int64_t nsteps)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (no_truth(m)) return MS_ERR_STATE;
    if (!(dt > 0.0) || !isfin(dt)) return fail(MS_ERR_ARG, "dt must be positive and finite");
    if (nsteps < 0) return fail(MS_ERR_ARG, "nsteps < 0");
    if (m->truth_dt == 0.0) m->truth_dt = dt;
    else if (dt != m->truth_dt) return fail(MS_ERR_ARG, "dt differs from the truth model's dt");
    Trace tr("msdem.truth steps");
    for (long long k = 0; k < nsteps; k++) {
        CK(truth_one(m, m->tcur, 1 - m->tcur, m->truth_steps));
        m->tcur = 1 - m->tcur;
        m->truth_steps++;
    }
    return read_errors(m);
}

int ms_truth_moments(ms_model *m, double *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    if (no_truth(m)) return MS_ERR_STATE;
    TruthArgs a;
    a.n = m->n;
    a.g = m->g;
    a.k = geo32(m->g.Lx, m->g.Ly, 1, 1, m->truth_dt > 0 ? m->truth_dt : 1.0);
    a.dt = m->truth_dt;
    a.step = m->truth_steps;
    a.ctrl = m->d_ctrl;
    a.fd = m->d_fd;
    if (m->precision == MS_FP64) CK(launch_truth_moments64(m->t64[m->tcur], m->P64, a, m->cb, m->d_tmom, m->stream));
    else CK(launch_truth_moments32(m->t32[m->tcur], m->P32, a, m->cb, m->d_tmom, m->stream));
    double *st = (double *)stage(m, sizeof(double) * m->ncell * NMOM);
    if (!st) return fail(MS_ERR_CUDA, "cudaMallocHost failed");
    CK(cudaMemcpyAsync(st, m->d_tmom, sizeof(double) * m->ncell * NMOM, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    std::memcpy(out, st, sizeof(double) * m->ncell * NMOM);
    return MS_OK;
}

static int ensure_scratch(ms_model *m)
{
    if (m->precision == MS_FP64) {
        if (!m->x64.x) CK(alloc64(m, m->x64, m->n));
        // radius is read-only except on update steps; keep the scratch copy valid
        CK(cudaMemcpyAsync(m->x64.r, m->s64.r, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->x64.h, m->s64.h, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
    } else {
        if (!m->x32.xq) {
            CK(alloc32(m, m->x32, m->n));
            CK(alloc_lists(m, m->xnl, m->n, m->ncell));
        }
        CK(cudaMemcpyAsync(m->x32.r, m->s32.r, sizeof(float) * m->n, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->x32.h, m->s32.h, sizeof(float) * m->n, cudaMemcpyDeviceToDevice, m->stream));
    }
    CK(cudaMemcpyAsync(m->d_xwin, m->d_win, sizeof(double) * m->ncell * NWIN, cudaMemcpyDeviceToDevice, m->stream));
    return MS_OK;
}

int ms_time_kernel(ms_model *m, int32_t which, double dt, int32_t reps, double *mean_ms)
{
    if (!m || !mean_ms) return fail(MS_ERR_ARG, "NULL argument");
    if (reps < 1) return fail(MS_ERR_ARG, "reps < 1");
    if (!(dt > 0.0)) return fail(MS_ERR_ARG, "dt must be positive");
    if (which == 1 && no_truth(m)) return MS_ERR_STATE;
    if (which < 0 || which > 2) return fail(MS_ERR_ARG, "which must be 0, 1 or 2");
    const double saved = m->dt, tsaved = m->truth_dt;
    int rc = ensure_scratch(m);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    m->dt = dt;
    m->truth_dt = dt;
    cudaError_t le = cudaSuccess;
    const long long i_local = m->steps % m->interval;
    // one warm-up launch, then the timed ones
    for (int k = 0; k <= reps && le == cudaSuccess; k++) {
        if (k == 1) le = cudaEventRecord(e0, m->stream);
        if (le != cudaSuccess) break;
        if (which == 0) le = launch_step(m, i_local, true);
        else if (which == 2 && interval_cells(m)) le = launch_interval_cells(m, true);
        else if (which == 2)
            for (int i = 0; i < m->interval && le == cudaSuccess; i++) le = launch_step(m, i, true);
        else le = truth_one(m, m->tcur, 1 - m->tcur, m->truth_steps);
    }
    if (le == cudaSuccess) le = cudaEventRecord(e1, m->stream);
    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->dt = saved;
    m->truth_dt = tsaved;
    if (le != cudaSuccess) return fail(MS_ERR_CUDA, "kernel timing failed: %s", cudaGetErrorString(le));
    *mean_ms = (double)ms / reps;
    return read_errors(m);
}

int ms_autotune(ms_model *m, double dt, int32_t reps, double *best_ms)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (reps < 1) return fail(MS_ERR_ARG, "reps < 1");
    std::vector<CellLaunch> cand;
    const int threads[3] = {64, 128, 256};
    for (int p = 0; p < 2; p++)
        for (int t : threads) {
            CellLaunch c = m->cl;
            c.variant = 0;
            c.threads = t;
            c.persistent = p;
            int per_sm = 2048 / t;
            c.grid = m->sm_count * std::min(per_sm, 8);
            cand.push_back(c);
        }
    if (m->precision == MS_FP32) {
        const float betas[5] = {0.6f, 0.8f, 1.0f, 1.3f, 1.7f};
        for (float b : betas) {
            CellLaunch c = m->cl;
            c.variant = 1;
            c.bin_beta = b;
            cand.push_back(c);
        }
        for (int v = 2; v <= 4; v++)
            for (float b : betas) {
                CellLaunch c = m->cl;
                c.variant = v;
                c.bin_beta = b;
                cand.push_back(c);
            }
        // variant 5: bins per cell, the skin's horizon and the floes per
        // block of small cells (how many cells share a block)
        const float skins[4] = {16.0f, 24.0f, 32.0f, 48.0f};
        const int caps[3] = {160, 208, RUN_T};
        for (float b : {1.0f, 1.3f, 1.7f})
            for (float sk : skins)
                for (int cap : caps) {
                    CellLaunch c = m->cl;
                    c.variant = 5;
                    c.bin_beta = b;
                    c.run_skin = sk;
                    c.run_cap1 = cap;
                    cand.push_back(c);
                }
    }
    // FP32: whole coarse intervals, so that variants that keep a cell
    // resident across steps are timed by what they save
    const int which = m->precision == MS_FP32 ? 2 : 0;
    const double per = which == 2 ? (double)m->interval : 1.0;
    const CellLaunch keep = m->cl;
    double best = 1e30;
    CellLaunch bestc = keep;
    for (const CellLaunch &c : cand) {
        if (configure_launch(m, c)) continue;
        double t = 0.0;
        if (ms_time_kernel(m, which, dt, reps, &t)) continue;
        t /= per;
        if (t < best) {
            best = t;
            bestc = c;
        }
    }
    int rc = configure_launch(m, best < 1e30 ? bestc : keep);
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    return MS_OK;
}

int ms_set_launch(ms_model *m, int32_t variant, int32_t threads, int32_t persistent, double bin_beta)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (variant != 0 && !((variant >= 1 && variant <= 5) && m->precision == MS_FP32))
        return fail(MS_ERR_ARG, "unsupported variant %d", variant);
    if (threads != 64 && threads != 128 && threads != 256) return fail(MS_ERR_ARG, "threads must be 64, 128 or 256");
    if (!(bin_beta > 0.1 && bin_beta < 10.0)) return fail(MS_ERR_ARG, "bin_beta must be in (0.1, 10)");
    CellLaunch c = m->cl;
    c.variant = variant;
    c.threads = threads;
    c.persistent = persistent ? 1 : 0;
    c.bin_beta = (float)bin_beta;
    c.grid = m->sm_count * std::min(2048 / threads, 8);
    CK(cudaStreamSynchronize(m->stream));
    return configure_launch(m, c);
}

int ms_info(ms_model *m, int64_t *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    Ctrl c;
    CK(cudaMemcpyAsync(&c, m->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    out[0] = m->n;
    out[1] = m->ncell;
    out[2] = m->max_n;
    out[3] = m->precision;
    out[4] = m->cl.variant;
    out[5] = m->cl.threads;
    out[6] = (int64_t)std::lround(m->cl.bin_beta * 1000.0f);
    out[7] = interval_launches(m);
    out[8] = m->fc.couple ? coarse_launches() : 1;
    out[9] = truth_launches(m->tb);
    out[10] = m->steps;
    out[11] = m->truth_steps;
    out[12] = m->replays;
    out[13] = (int64_t)c.deep;
    out[14] = m->cl.persistent;
    out[15] = c.N1;
    out[16] = (int64_t)std::lround(m->cl.run_skin * 1000.0f);
    out[17] = m->cl.run_cap1;
    out[18] = m->shard_nranks;
    out[19] = m->shard_rank;
    out[20] = m->shard_nranks ? m->shard_nown : m->ncell;
    return MS_OK;
}

int ms_set_resident(ms_model *m, double skin_steps, int32_t block_floes)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (!(skin_steps >= 1.0 && skin_steps <= 1000.0)) return fail(MS_ERR_ARG, "skin_steps must be in [1, 1000]");
    if (block_floes < 32 || block_floes > RUN_T)
        return fail(MS_ERR_ARG, "block_floes must be in [32, %d]", RUN_T);
    CellLaunch c = m->cl;
    c.run_skin = (float)skin_steps;
    c.run_cap1 = block_floes;
    CK(cudaStreamSynchronize(m->stream));
    return configure_launch(m, c);
}

int ms_floe_cells(const ms_grid *grid, const ms_floes *floes, int32_t *cell_out)
{
    if (!grid || !cell_out) return fail(MS_ERR_ARG, "NULL argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nens < 0 || grid->nens > 65536 || !(grid->Lx > 0.0) ||
        !(grid->Ly > 0.0) || !isfin(grid->Lx) || !isfin(grid->Ly))
        return fail(MS_ERR_ARG, "bad grid");
    int rc = check_floe_args(floes, -1);
    if (rc) return rc;
    const long long n = floes->n;
    const long long l = host_first(n, [&](long long k) { return !isfin(floes->x[k]) || !isfin(floes->y[k]); });
    if (l < n) return fail(MS_ERR_ARG, "floe %lld has a non-finite position", l);
    if (n == 0) return MS_OK;
    // the kernel ms_init assigns cells with, on the current device
    const Geom g = grid_geom(grid);
    UpGeom ug{n, g.nx, g.ny, g.Lx, g.Ly, g.Lcx, g.Lcy};
    double *xy = nullptr;
    int *cell = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&xy, sizeof(double) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc(&cell, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(xy, floes->x, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(xy + n, floes->y, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_cell_of(xy, ug, cell, nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cell_out, cell, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(xy);
    cudaFree(cell);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(MS_ERR_CUDA, "cell assignment failed: %s", cudaGetErrorString(e));
    return MS_OK;
}

int ms_layout(ms_model *m, int32_t *off, int32_t *orig)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (off) std::copy(m->h_off.begin(), m->h_off.end(), off);
    if (orig)
        for (long long k = 0; k < m->n; k++) orig[k] = (int32_t)m->h_orig[k];
    return MS_OK;
}

int ms_set_shard(ms_model *m, int32_t nranks, int32_t rank, const int32_t *rank_off, const int32_t *cells,
                 ms_exchange_fn fn, void *ctx)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (m->shard_nranks) return fail(MS_ERR_STATE, "the model is already sharded");
    if (m->hybrid_mode >= 0) return fail(MS_ERR_STATE, "a model with a closure attached cannot be sharded");
    if (!rank_off || !cells || !fn) return fail(MS_ERR_ARG, "NULL argument");
    if (nranks < 1 || rank < 0 || rank >= nranks) return fail(MS_ERR_ARG, "need 0 <= rank < nranks");
    const int nc = m->ncell;
    if (rank_off[0] != 0 || rank_off[nranks] != nc) return fail(MS_ERR_ARG, "rank_off must run from 0 to %d", nc);
    int maxc = 0;
    for (int r = 0; r < nranks; r++) {
        if (rank_off[r + 1] < rank_off[r]) return fail(MS_ERR_ARG, "rank_off decreases at rank %d", r);
        maxc = std::max(maxc, rank_off[r + 1] - rank_off[r]);
    }
    std::vector<int> seen(nc, -1);
    std::vector<long long> rows(nc);
    for (int r = 0; r < nranks; r++)
        for (int t = rank_off[r]; t < rank_off[r + 1]; t++) {
            const int c = cells[t];
            if (c < 0 || c >= nc || seen[c] >= 0) return fail(MS_ERR_ARG, "cells is not a permutation of the cells");
            seen[c] = r;
            rows[t] = (long long)r * maxc + (t - rank_off[r]);
        }
    for (int c = 0; c < nc; c++)
        if (seen[c] != rank && m->h_off[c + 1] > m->h_off[c])
            return fail(MS_ERR_ARG, "cell %d holds floes but belongs to rank %d", c, seen[c]);
    CK(cudaStreamSynchronize(m->stream));
    const size_t ncol = SHARD_NCOL;
    if (dalloc(m, &m->d_shard_cells, nc) != cudaSuccess || dalloc(m, &m->d_shard_rows, nc) != cudaSuccess ||
        dalloc(m, &m->d_send, (size_t)std::max(maxc, 1) * ncol) != cudaSuccess ||
        dalloc(m, &m->d_recv, (size_t)nranks * std::max(maxc, 1) * ncol) != cudaSuccess)
        return fail(MS_ERR_CUDA, "cudaMalloc of the exchange buffers failed");
    CK(cudaMemcpyAsync(m->d_shard_cells, cells, sizeof(int) * nc, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemcpyAsync(m->d_shard_rows, rows.data(), sizeof(long long) * nc, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemsetAsync(m->d_send, 0, sizeof(double) * std::max(maxc, 1) * ncol, m->stream));
    CK(cudaMemsetAsync(m->d_recv, 0, sizeof(double) * nranks * std::max(maxc, 1) * ncol, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    drop_graph(m);
    m->shard_nranks = nranks;
    m->shard_rank = rank;
    m->shard_first = rank_off[rank];
    m->shard_nown = rank_off[rank + 1] - rank_off[rank];
    m->shard_maxc = maxc;
    m->exch = fn;
    m->exch_ctx = ctx;
    return MS_OK;
}

int ms_shard_buffers(ms_model *m, double **send, double **recv, int32_t *max_cells)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (!m->shard_nranks) return fail(MS_ERR_STATE, "the model is not sharded");
    if (send) *send = m->d_send;
    if (recv) *recv = m->d_recv;
    if (max_cells) *max_cells = m->shard_maxc;
    return MS_OK;
}

int ms_cell_moments_noalloc(const ms_grid *grid, double rho_ice, int32_t inertia_half, int64_t n,
                            const double *x, const double *y, const double *u, const double *v,
                            const double *omega, const double *r, const double *h, const double *fd,
                            double *out, void *stream)
{
    if (!grid) return fail(MS_ERR_ARG, "grid is NULL");
    if (grid->nx < 1 || grid->ny < 1 || !(grid->Lx > 0.0) || !(grid->Ly > 0.0) || !isfin(grid->Lx) ||
        !isfin(grid->Ly))
        return fail(MS_ERR_ARG, "grid needs nx, ny >= 1 and positive finite sides");
    if (grid->nens < 0) return fail(MS_ERR_ARG, "nens must be >= 0");
    const int nens = grid->nens > 1 ? grid->nens : 1;
    if ((long long)grid->nx * grid->ny * nens > noalloc_max_cells())
        return fail(MS_ERR_ARG, "ms_cell_moments_noalloc handles at most %d cells, got %lld", noalloc_max_cells(),
                    (long long)grid->nx * grid->ny * nens);
    if (n < 0 || n > noalloc_max_floes())
        return fail(MS_ERR_ARG, "ms_cell_moments_noalloc handles 0 to %lld floes, got %lld", noalloc_max_floes(),
                    (long long)n);
    if (!(rho_ice > 0.0) || !isfin(rho_ice)) return fail(MS_ERR_ARG, "rho_ice must be positive");
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    if (n > 0 && (!x || !y || !u || !v || !omega || !r || !h || !fd)) return fail(MS_ERR_ARG, "a floe array is NULL");
    Geom g;
    g.nx = grid->nx;
    g.ny = grid->ny * nens;
    g.nyr = grid->ny;
    g.nens = nens;
    g.Lx = grid->Lx;
    g.Ly = grid->Ly * nens;
    g.Lcx = grid->Lx / grid->nx;
    g.Lcy = grid->Ly / grid->ny;
    cudaStream_t st = (cudaStream_t)stream;
    CK(noalloc_cell_moments(g, rho_ice * PI_D, inertia_half ? 0.5 : 1.0, n, x, y, u, v, omega, r, h, fd, out, st));
    CK(cudaStreamSynchronize(st));
    return MS_OK;
}

int ms_closure_attach(ms_model *m, ms_mlp *mlp, int32_t mode, double tol, const float *box)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (mode < -1 || mode > 2) return fail(MS_ERR_ARG, "mode must be -1, 0, 1 or 2");
    if ((mode == 0 || mode == 2) && !mlp) return fail(MS_ERR_ARG, "modes 0 and 2 need a network");
    if (mode >= 0 && (m->precision != MS_FP32 || !m->fc.couple))
        return fail(MS_ERR_STATE, "the closure runs on coupled FP32 models");
    if (mode >= 0 && m->shard_nranks) return fail(MS_ERR_STATE, "a sharded model runs no closure");
    if (!(tol >= 0.0)) return fail(MS_ERR_ARG, "tol must be >= 0");
    if (mode >= 0 && m->steps % m->interval != 0) return fail(MS_ERR_STATE, "attach between coarse intervals");
    CK(cudaStreamSynchronize(m->stream));
    const int nc = m->ncell;
    if (!m->d_X) {
        CK(dalloc(m, &m->d_X, (size_t)nc * NFEAT));
        CK(dalloc(m, &m->d_Ylag, (size_t)nc * 4));
        CK(dalloc(m, &m->d_nerr, nc));
        CK(dalloc(m, &m->d_age, nc));
        CK(dalloc(m, &m->d_Yp, (size_t)nc * 4));
        CK(dalloc(m, &m->d_Yuse, (size_t)nc * 4));
        CK(dalloc(m, &m->d_Yc, (size_t)nc * 4));
        CK(dalloc(m, &m->d_box, 2 * NFEAT));
        CK(dalloc(m, &m->d_isc, nc));
        CK(dalloc(m, &m->d_order2, nc));
        CK(dalloc(m, &m->d_live, MAXSEG));
        CK(dalloc(m, &m->d_ocean, (size_t)nc * 4));
        CK(launch_ocean_at_centres(nc, m->g, m->P64, m->d_ocean, m->stream));
        CK(dalloc(m, &m->d_segb, MAXSEG));
        CK(dalloc(m, &m->d_sege, MAXSEG));
        CK(dalloc(m, &m->d_mom0, (size_t)nc * NMOM));
        CK(dalloc(m, &m->d_ccount, 1));
        CK(cudaMemsetAsync(m->d_ccount, 0, sizeof(unsigned long long), m->stream));
    }
    float hb[2 * NFEAT];
    for (int k = 0; k < NFEAT; k++) {
        hb[k] = box ? box[k] : -3.0e38f;
        hb[NFEAT + k] = box ? box[NFEAT + k] : 3.0e38f;
    }
    CK(cudaMemcpyAsync(m->d_box, hb, sizeof(hb), cudaMemcpyHostToDevice, m->stream));
    // no cell has been checked yet: every cell's first interval runs its DEM
    {
        std::vector<float> big(nc, 3.0e38f);
        CK(cudaMemcpyAsync(m->d_nerr, big.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemsetAsync(m->d_age, 0, sizeof(int) * nc, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    const int prev_mode = m->hybrid_mode;
    m->hybrid_mode = mode;
    m->mlp = mlp;
    m->hybrid_tol = tol;
    CellLaunch cl = m->cl;
    if (mode >= 0 && cl.variant == 0) cl.variant = 2;
    int rc = configure_launch(m, cl);
    if (rc) {
        m->hybrid_mode = prev_mode;
        return rc;
    }
    drop_graph(m);
    CK(cudaStreamSynchronize(m->stream));
    return MS_OK;
}

int ms_closure_collect(ms_model *m, int32_t nint, float *X, float *Y)
{
    if (!m || !X || !Y) return fail(MS_ERR_ARG, "NULL argument");
    if (nint < 1) return fail(MS_ERR_ARG, "nint must be >= 1");
    if (!m->fc.couple || m->precision != MS_FP32) return fail(MS_ERR_STATE, "collect runs on coupled FP32 models");
    if (m->shard_nranks) return fail(MS_ERR_STATE, "a sharded model runs no closure");
    if (m->dt == 0.0) return fail(MS_ERR_STATE, "step the model once first (dt is not set)");
    if (m->steps % m->interval != 0) return fail(MS_ERR_STATE, "collect starts between coarse intervals");
    if (!m->d_X) {
        int rc = ms_closure_attach(m, nullptr, -1, 0.0, nullptr);
        if (rc) return rc;
    }
    const int saved = m->hybrid_mode;
    m->hybrid_mode = -1;
    const int nc = m->ncell;
    const double dT = (double)m->fc.N0 * m->dt;
    int rc = MS_OK;
    // the lagged features need the tendencies of the interval before: without
    // them, run one interval first and return only the ones after it
    Ctrl c0;
    CK(cudaMemcpyAsync(&c0, m->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    const int first = (c0.lag_mark == c0.base + 1) ? 0 : -1;
    for (int k = first; k < nint && rc == MS_OK; k++) {
        cudaError_t e = cudaMemcpyAsync(m->d_mom0, m->d_mom, sizeof(double) * nc * NMOM, cudaMemcpyDeviceToDevice,
                                        m->stream);
        if (e == cudaSuccess)
            e = launch_features(m->d_mom, m->d_tgt, nc, m->g, m->P64, m->d_ctrl, m->dt, m->fc.N0, m->fc.n_t,
                                m->d_Ylag, m->d_ocean, m->d_X, m->stream);
        if (e == cudaSuccess && interval_cells(m)) e = launch_interval_cells(m, false);
        else
            for (int i = 0; i < m->interval && e == cudaSuccess; i++) e = launch_step(m, i, false);
        if (e == cudaSuccess)
            e = launch_collect_targets(m->d_mom0, m->d_mom, m->d_win, nc, m->fc.N0, dT, nullptr, nullptr, m->d_ctrl,
                                       m->d_Ylag, m->d_Yc, nullptr, 0.0, nullptr, nullptr, m->stream);
        if (e == cudaSuccess) e = launch_interval_end(m);
        if (e == cudaSuccess && k >= 0)
            e = cudaMemcpyAsync(X + (size_t)k * nc * NFEAT, m->d_X, sizeof(float) * nc * NFEAT,
                                cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess && k >= 0)
            e = cudaMemcpyAsync(Y + (size_t)k * nc * 4, m->d_Yc, sizeof(float) * nc * 4, cudaMemcpyDeviceToHost,
                                m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) rc = fail(MS_ERR_CUDA, "collect failed: %s", cudaGetErrorString(e));
        m->steps += m->interval;
    }
    m->hybrid_mode = saved;
    if (rc) return rc;
    return read_errors(m);
}

int ms_closure_stats(ms_model *m, int64_t *out)
{
    if (!m || !out) return fail(MS_ERR_ARG, "NULL argument");
    unsigned long long cc = 0;
    if (m->d_ccount) {
        CK(cudaMemcpyAsync(&cc, m->d_ccount, sizeof(cc), cudaMemcpyDeviceToHost, m->stream));
    }
    CK(cudaStreamSynchronize(m->stream));
    out[0] = (int64_t)cc;
    out[1] = m->ncell;
    out[2] = m->hybrid_mode;
    out[3] = m->steps / m->interval;
    return MS_OK;
}

}  // extern "C"
