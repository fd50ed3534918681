// upload.cu -- the caller's floes into the cell layout, on the device.
//
// The host copies the eight FP64 input arrays into pinned memory (all cores)
// and from there to the device in one transfer; these kernels assign the
// floes to cells, check them and write the stored state, one thread per
// floe.  The arithmetic is written with explicitly rounded operations (no
// contraction into FMAs), so the assignment is the plain IEEE evaluation of
// X - L floor(X / L) and floor(X / d) wherever it runs.
#include "upload.cuh"

namespace msd {

namespace {

constexpr int UP_T = 256;

// X wrapped into [0, L) the way the host does it: X - L floor(X / L)
__device__ __forceinline__ double wrap_d(double X, double L)
{
    return __dsub_rn(X, __dmul_rn(L, floor(__ddiv_rn(X, L))));
}

__device__ __forceinline__ int cell_index_d(double X, double L, double d, int n)
{
    int i = (int)floor(__ddiv_rn(wrap_d(X, L), d));
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    return i;
}

// fraction of the cell -> 32-bit fixed point (2^32 == 1, wraps); round to
// nearest, ties to even, as the host's nearbyint in the default mode
__device__ __forceinline__ uint32_t to_fix_d(double frac)
{
    const long long iv = (long long)rint(__dmul_rn(frac, 4294967296.0));
    return (uint32_t)(iv & 0xffffffffLL);
}

__global__ void __launch_bounds__(UP_T) k_check_floes(const double *__restrict__ raw,
                                                      const int *__restrict__ cell_of, UpGeom g,
                                                      unsigned long long *first)
{
    const long long n = g.n;
    for (long long l = blockIdx.x * (long long)UP_T + threadIdx.x; l < n; l += (long long)gridDim.x * UP_T) {
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 8; a++) ok &= isfinite(raw[a * n + l]);
        ok &= raw[6 * n + l] > 0.0 && raw[7 * n + l] > 0.0;
        if (!ok) {
            atomicMin(&first[0], (unsigned long long)l);
            continue;
        }
        const int c = cell_index_d(raw[n + l], g.Ly, g.Lcy, g.ny) * g.nx + cell_index_d(raw[l], g.Lx, g.Lcx, g.nx);
        if (c != cell_of[l]) atomicMin(&first[1], (unsigned long long)l);
    }
}

__global__ void __launch_bounds__(UP_T) k_floes_to_cells32(const double *__restrict__ raw,
                                                           const int *__restrict__ orig,
                                                           const int *__restrict__ cell_of, UpGeom g, DevState32 s)
{
    const long long n = g.n;
    for (long long k = blockIdx.x * (long long)UP_T + threadIdx.x; k < n; k += (long long)gridDim.x * UP_T) {
        const long long l = orig[k];
        const int c = cell_of[l];
        const int ix = c % g.nx, iy = c / g.nx;
        const double Xw = wrap_d(raw[l], g.Lx), Yw = wrap_d(raw[n + l], g.Ly);
        s.xq[k] = to_fix_d(__ddiv_rn(__dsub_rn(Xw, __dmul_rn((double)ix, g.Lcx)), g.Lcx));
        s.yq[k] = to_fix_d(__ddiv_rn(__dsub_rn(Yw, __dmul_rn((double)iy, g.Lcy)), g.Lcy));
        s.th[k] = __double2float_rn(raw[2 * n + l]);
        s.u[k] = __double2float_rn(raw[3 * n + l]);
        s.v[k] = __double2float_rn(raw[4 * n + l]);
        s.w[k] = __double2float_rn(raw[5 * n + l]);
        s.r[k] = __double2float_rn(raw[6 * n + l]);
        s.h[k] = __double2float_rn(raw[7 * n + l]);
    }
}

__global__ void __launch_bounds__(UP_T) k_floes_to_cells64(const double *__restrict__ raw,
                                                           const int *__restrict__ orig,
                                                           const int *__restrict__ cell_of, UpGeom g, DevState64 s)
{
    const long long n = g.n;
    for (long long k = blockIdx.x * (long long)UP_T + threadIdx.x; k < n; k += (long long)gridDim.x * UP_T) {
        const long long l = orig[k];
        const int c = cell_of[l];
        const int ix = c % g.nx, iy = c / g.nx;
        s.x[k] = __dsub_rn(wrap_d(raw[l], g.Lx), __dmul_rn((double)ix, g.Lcx));
        s.y[k] = __dsub_rn(wrap_d(raw[n + l], g.Ly), __dmul_rn((double)iy, g.Lcy));
        s.th[k] = raw[2 * n + l];
        s.u[k] = raw[3 * n + l];
        s.v[k] = raw[4 * n + l];
        s.w[k] = raw[5 * n + l];
        s.r[k] = raw[6 * n + l];
        s.h[k] = raw[7 * n + l];
    }
}

// the cell of every caller floe (and the count of each cell)
__global__ void __launch_bounds__(UP_T) k_cell_of(const double *__restrict__ raw, UpGeom g, int *__restrict__ cell_of,
                                                  int *__restrict__ count)
{
    const long long n = g.n;
    for (long long l = blockIdx.x * (long long)UP_T + threadIdx.x; l < n; l += (long long)gridDim.x * UP_T) {
        const int c = cell_index_d(raw[n + l], g.Ly, g.Lcy, g.ny) * g.nx + cell_index_d(raw[l], g.Lx, g.Lcx, g.nx);
        cell_of[l] = c;
        if (count) atomicAdd(&count[c], 1);
    }
}

// one thread per floe, at most 65,536 blocks (a grid-stride loop covers the rest)
int up_blocks(long long n)
{
    const long long b = (n + UP_T - 1) / UP_T;
    return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

cudaError_t launch_cell_of(const double *raw, UpGeom g, int *cell_of, int *count, cudaStream_t st)
{
    if (g.n == 0) return cudaSuccess;
    k_cell_of<<<up_blocks(g.n), UP_T, 0, st>>>(raw, g, cell_of, count);
    return cudaGetLastError();
}

cudaError_t launch_check_floes(const double *raw, const int *cell_of, UpGeom g, unsigned long long *first,
                               cudaStream_t st)
{
    if (g.n == 0) return cudaSuccess;
    k_check_floes<<<up_blocks(g.n), UP_T, 0, st>>>(raw, cell_of, g, first);
    return cudaGetLastError();
}

cudaError_t launch_floes_to_cells32(const double *raw, const int *orig, const int *cell_of, UpGeom g,
                                    DevState32 s, cudaStream_t st)
{
    if (g.n == 0) return cudaSuccess;
    k_floes_to_cells32<<<up_blocks(g.n), UP_T, 0, st>>>(raw, orig, cell_of, g, s);
    return cudaGetLastError();
}

cudaError_t launch_floes_to_cells64(const double *raw, const int *orig, const int *cell_of, UpGeom g,
                                    DevState64 s, cudaStream_t st)
{
    if (g.n == 0) return cudaSuccess;
    k_floes_to_cells64<<<up_blocks(g.n), UP_T, 0, st>>>(raw, orig, cell_of, g, s);
    return cudaGetLastError();
}

}  // namespace msd
