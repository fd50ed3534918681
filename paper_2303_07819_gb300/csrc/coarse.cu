// coarse.cu -- the coarse step of Algorithm 1 in FP64: process the window of
// DEM data, solve the moment equations by Lax-Friedrichs with N1 substeps, and
// set the targets of the gradual update.
//
// Moment equations, Eq. (2.26a-c): rho and P_omega in conservative form; rho v
// in the Oseen form <v> . grad(rho v) of Eq. (3.3).  reading: 2-D LF with the
// four-neighbour average on the periodic grid, <v> = window mean of the cell's
// mass-weighted velocity, drag sources = window mean of the cell's total drag
// per unit area; N1 = max(1, ceil(dT max|V|/dX / 0.5)) (Sec. 3.2).
// Walls (Sec. 4.4): the neighbours beyond x = 0 and x = Lx are ghost cells;
// walls = 1, zero Dirichlet as the paper states it: the ghost's fields, and so
// its fluxes, are zero; walls = 2, impermeable: the ghost mirrors the boundary
// cell (rho, rho v_y, P_omega equal; rho v_x and <v_x> of opposite sign), so
// no mass crosses the wall.
//
// N1 is chosen on the device (it depends on the window data).  The step is
// one cooperative launch whose blocks pass each phase (prepare, the N1
// substeps, targets, finish) together with grid-wide barriers between them,
// so it fits a CUDA graph as a single node; a device that cannot hold the
// cooperative grid takes the phases as a fixed sequence of launches (NSUB_MAX
// substeps that return at once past N1).
#include <cooperative_groups.h>

#include "common.cuh"
#include "shard.cuh"

namespace cg = cooperative_groups;

namespace msd {

namespace {

// substeps of realization e (each realization of an ensemble is its own
// coarse problem, so each takes its own N1)
__device__ __forceinline__ int n_sub(const CoarseArgs &a, int e)
{
    const double cmax = __longlong_as_double((long long)a.cmax[e]);
    int N1 = (int)ceil(a.dT * cmax / 0.5);
    return N1 < 1 ? 1 : N1;
}

__device__ __forceinline__ void coarse_prepare_cell(const CoarseArgs &a, int c)
{
    const int nc = a.nx * a.ny;
    const double *mo = a.mom + (size_t)c * NMOM;
    if (!a.ctrl->have_q) {
        // initialise the coarse model from the DEM data (Sec. 3.2)
        a.q0[c] = mo[1] / a.Ac;
        a.q0[nc + c] = mo[2] / a.Ac;
        a.q0[2 * nc + c] = mo[3] / a.Ac;
        a.q0[3 * nc + c] = mo[5] / a.Ac;
    }
    const double N0 = (double)a.N0;
    const double Vx = a.win[c] / N0, Vy = a.win[nc + c] / N0;
    a.V[c] = Vx;
    a.V[nc + c] = Vy;
    a.S[c] = 0.0;
    a.S[nc + c] = a.win[2 * nc + c] / N0 / a.Ac;
    a.S[2 * nc + c] = a.win[3 * nc + c] / N0 / a.Ac;
    a.S[3 * nc + c] = a.win[4 * nc + c] / N0 / a.Ac;
    for (int k = 0; k < NWIN; k++) a.win[k * nc + c] = 0.0;
    const double cx = fabs(Vx) / a.dx, cy = fabs(Vy) / a.dy;
    const double cc = cx > cy ? cx : cy;
    atomicMax(&a.cmax[c / (a.nx * a.nyr)], (unsigned long long)__double_as_longlong(cc));
}

__device__ __forceinline__ void coarse_lf_cell(const CoarseArgs &a, int k, int c)
{
    const int nx = a.nx, ny = a.nyr, nc = nx * a.ny;
    const int e = c / (nx * ny);
    const int N1 = n_sub(a, e);
    if (k >= N1) return;
    const double *q = (k & 1) ? a.q1 : a.q0;
    double *qn = (k & 1) ? a.q0 : a.q1;
    const double dtau = a.dT / N1;
    const int i = c % nx, j = (c / nx) % ny, b = e * nx * ny;   // b: the realization's first cell
    const int cE = b + j * nx + (i + 1) % nx, cW = b + j * nx + (i + nx - 1) % nx;
    const int cN = b + ((j + 1) % ny) * nx + i, cS = b + ((j + ny - 1) % ny) * nx + i;
    const double *Vx = a.V, *Vy = a.V + nc;
    const bool ghE = a.walls && i == nx - 1, ghW = a.walls && i == 0;
    const bool mirror = a.walls == 2;
#pragma unroll
    for (int f = 0; f < 4; f++) {
        const double *g = q + (size_t)f * nc;
        // the ghost's field and <v_x>
        const double gG = mirror ? (f == 1 ? -g[c] : g[c]) : 0.0, VG = mirror ? -Vx[c] : 0.0;
        const double gE = ghE ? gG : g[cE], gW = ghW ? gG : g[cW];
        const double VE = ghE ? VG : Vx[cE], VW = ghW ? VG : Vx[cW];
        const double avg = 0.25 * ((gE + gW) + (g[cN] + g[cS]));
        double val;
        if (f == 0 || f == 3) {
            val = avg - dtau / (2.0 * a.dx) * (VE * gE - VW * gW)
                      - dtau / (2.0 * a.dy) * (Vy[cN] * g[cN] - Vy[cS] * g[cS]);
        } else {
            val = avg - dtau * Vx[c] / (2.0 * a.dx) * (gE - gW)
                      - dtau * Vy[c] / (2.0 * a.dy) * (g[cN] - g[cS]);
        }
        qn[(size_t)f * nc + c] = val + dtau * a.S[(size_t)f * nc + c];
    }
}

// Targets of the gradual update (Sec. 3.3).  reading: the radius scale s
// makes the cell mass equal rho* A_c; the uniform velocity and spin increments
// make the scaled cell's momentum and angular momentum equal the coarse ones.
__device__ __forceinline__ void coarse_targets_cell(const CoarseArgs &a, int c)
{
    const int nc = a.nx * a.ny;
    const int N1 = n_sub(a, c / (a.nx * a.nyr));
    const double *q = ((N1 < NSUB_MAX ? N1 : NSUB_MAX) & 1) ? a.q1 : a.q0;
    double qc[4];
    for (int f = 0; f < 4; f++) {
        qc[f] = q[(size_t)f * nc + c];
        if (q != a.q0) a.q0[(size_t)f * nc + c] = qc[f];
    }
    const double *mo = a.mom + (size_t)c * NMOM;
    const double M = mo[1];
    double s = 1.0, dvx = 0.0, dvy = 0.0, dw = 0.0;
    if (M > 0.0) {
        const double rho_dem = M / a.Ac;
        const double qr = qc[0] > 0.0 ? qc[0] : 0.0;
        s = sqrt(qr / rho_dem);
        const double s2 = s * s, s4 = s2 * s2;
        if (s2 * M > 0.0) {
            dvx = (qc[1] * a.Ac - s2 * mo[2]) / (s2 * M);
            dvy = (qc[2] * a.Ac - s2 * mo[3]) / (s2 * M);
        }
        if (s4 * mo[4] > 0.0) dw = (qc[3] * a.Ac - s4 * mo[5]) / (s4 * mo[4]);
    }
    a.tgt[c] = s;
    a.tgt[nc + c] = dvx;
    a.tgt[2 * nc + c] = dvy;
    a.tgt[3 * nc + c] = dw;
}

__device__ __forceinline__ void coarse_finish(const CoarseArgs &a)
{
    int N1 = 1;
    for (int e = 0; e < a.nens; e++) {
        const int n1 = n_sub(a, e);
        N1 = n1 > N1 ? n1 : N1;
        a.cmax[e] = 0ull;
    }
    Ctrl *ctrl = a.ctrl;
    ctrl->N1 = N1;      // the largest over the realizations
    if (N1 > NSUB_MAX) ctrl->err |= ERR_CFL;
    ctrl->have_q = 1;
    ctrl->have_tgt = 1;
    ctrl->base += a.N0;
}

// the phases as separate launches (a thread per cell)
__global__ void k_coarse_prepare(CoarseArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.nx * a.ny) coarse_prepare_cell(a, c);
}

__global__ void k_coarse_lf(CoarseArgs a, int k)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.nx * a.ny) coarse_lf_cell(a, k, c);
}

__global__ void k_coarse_targets(CoarseArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.nx * a.ny) coarse_targets_cell(a, c);
}

__global__ void k_coarse_finish(CoarseArgs a) { coarse_finish(a); }

// The whole coarse step in one cooperative launch: every block runs each
// phase over a grid-stride share of the cells, with a grid-wide barrier
// between phases (each substep reads the neighbours the one before wrote),
// and the substeps stop at the largest N1 of the realizations.
constexpr int CF_T = 256;

__global__ void __launch_bounds__(CF_T) k_coarse_fused(CoarseArgs a)
{
    cg::grid_group grid = cg::this_grid();
    const int nc = a.nx * a.ny;
    const int c0 = blockIdx.x * blockDim.x + threadIdx.x, cs = gridDim.x * blockDim.x;
    for (int c = c0; c < nc; c += cs) coarse_prepare_cell(a, c);
    grid.sync();
    // the largest substep count over the realizations (every block the same)
    __shared__ int n1s[CF_T / 32];
    int n1 = 1;
    for (int e = threadIdx.x; e < a.nens; e += CF_T) n1 = max(n1, n_sub(a, e));
    for (int d = 16; d > 0; d >>= 1) n1 = max(n1, __shfl_xor_sync(0xffffffffu, n1, d));
    if ((threadIdx.x & 31) == 0) n1s[threadIdx.x >> 5] = n1;
    __syncthreads();
    int n1max = 1;
    for (int w = 0; w < CF_T / 32; w++) n1max = max(n1max, n1s[w]);
    n1max = min(n1max, NSUB_MAX);
    for (int k = 0; k < n1max; k++) {
        for (int c = c0; c < nc; c += cs) coarse_lf_cell(a, k, c);
        grid.sync();
    }
    for (int c = c0; c < nc; c += cs) coarse_targets_cell(a, c);
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) coarse_finish(a);
}

__global__ void k_advance(Ctrl *ctrl, int N0) { ctrl->base += N0; }

// Sharded grids: the coarse step of a cell reads its moment columns 1-5 and
// its five window sums and nothing else of the DEM (k_coarse_prepare,
// k_coarse_targets).  A rank packs those of its own cells, row k of `send`
// for its k-th cell, and after the exchange writes every gathered row back
// into the cell it belongs to.
__global__ void k_shard_pack(const double *mom, const double *win, int nc, const int *cells, int ncells,
                             double *send)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    const int c = cells[k];
    double *o = send + (size_t)k * SHARD_NCOL;
    for (int a = 0; a < 5; a++) o[a] = mom[(size_t)c * NMOM + 1 + a];
    for (int a = 0; a < NWIN; a++) o[5 + a] = win[(size_t)a * nc + c];
}

__global__ void k_shard_scatter(double *mom, double *win, int nc, const int *cells, const long long *rows,
                                const double *recv)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int c = cells[t];
    const double *i = recv + (size_t)rows[t] * SHARD_NCOL;
    for (int a = 0; a < 5; a++) mom[(size_t)c * NMOM + 1 + a] = i[a];
    for (int a = 0; a < NWIN; a++) win[(size_t)a * nc + c] = i[5 + a];
}

}  // namespace

cudaError_t launch_shard_pack(const double *mom, const double *win, int nc, const int *cells, int ncells,
                              double *send, cudaStream_t st)
{
    if (ncells > 0) k_shard_pack<<<(ncells + 255) / 256, 256, 0, st>>>(mom, win, nc, cells, ncells, send);
    return cudaGetLastError();
}

cudaError_t launch_shard_scatter(double *mom, double *win, int nc, const int *cells, const long long *rows,
                                 const double *recv, cudaStream_t st)
{
    k_shard_scatter<<<(nc + 255) / 256, 256, 0, st>>>(mom, win, nc, cells, rows, recv);
    return cudaGetLastError();
}

int coarse_launches() { return 1; }

// grid of the fused coarse step: as many blocks as the device holds at once
// (a cooperative launch needs them all resident), at most one per 256 cells
static int coarse_fused_grid(int nc)
{
    static int per_sm = -1, nsm = 0;
    if (per_sm < 0) {
        int dev = 0, b = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_coarse_fused, CF_T, 0) != cudaSuccess) b = 0;
        per_sm = b;
    }
    const int need = (nc + CF_T - 1) / CF_T, most = per_sm * nsm;
    return need < most ? need : most;
}

cudaError_t launch_coarse_step(const CoarseArgs &a, cudaStream_t st)
{
    const int nc = a.nx * a.ny;
    const int G = coarse_fused_grid(nc);
    if (G > 0) {
        void *args[] = {const_cast<CoarseArgs *>(&a)};
        return cudaLaunchCooperativeKernel((const void *)k_coarse_fused, dim3(G), dim3(CF_T), args, 0, st);
    }
    // the phases launch by launch (a device that cannot hold a cooperative grid)
    const int T = 256, B = (nc + T - 1) / T;
    k_coarse_prepare<<<B, T, 0, st>>>(a);
    for (int k = 0; k < NSUB_MAX; k++) k_coarse_lf<<<B, T, 0, st>>>(a, k);
    k_coarse_targets<<<B, T, 0, st>>>(a);
    k_coarse_finish<<<1, 1, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance(Ctrl *ctrl, int N0, cudaStream_t st)
{
    k_advance<<<1, 1, 0, st>>>(ctrl, N0);
    return cudaGetLastError();
}

}  // namespace msd
