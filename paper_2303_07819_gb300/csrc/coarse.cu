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
// N1 is chosen on the device (it depends on the window data), so the step is
// a fixed sequence of launches (prepare, NSUB_MAX substeps that return at once
// past N1, targets, finish) and can be captured in a CUDA graph.
#include "common.cuh"
#include "shard.cuh"

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

__global__ void k_coarse_prepare(CoarseArgs a)
{
    const int nc = a.nx * a.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
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

__global__ void k_coarse_lf(CoarseArgs a, int k)
{
    const int nx = a.nx, ny = a.nyr, nc = nx * a.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
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
__global__ void k_coarse_targets(CoarseArgs a)
{
    const int nc = a.nx * a.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
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

__global__ void k_coarse_finish(CoarseArgs a)
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

int coarse_launches() { return NSUB_MAX + 3; }

cudaError_t launch_coarse_step(const CoarseArgs &a, cudaStream_t st)
{
    const int nc = a.nx * a.ny;
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
