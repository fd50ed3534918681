// fixsum.cuh -- exact per-cell sums of FP32 values, whatever the order.
//
// A value v of a (cell, column) whose largest magnitude lies in [2^e,
// 2^(e + 1)) counts as the integer round(v 2^(FIX_SHIFT - e)), at most 2^50
// in magnitude, so up to 4096 values sum exactly in 64 bits; the total
// converts back once.  Values below 2^(e - FIX_SHIFT) round to the nearest
// multiple of it, far below FP32 resolution of the total.  Integer sums do
// not depend on the order of addition, so a cell's sums are the same however
// its floes are distributed over threads, warps and blocks.
#pragma once
#include <cuda_runtime.h>

namespace msd {

constexpr int FIX_SHIFT = 49;
constexpr int FIX_NONE = -30000;   // exponent of a column with no nonzero value

// a value counts if it is finite and nonzero
__device__ __forceinline__ float fix_counted(float x) { return (x != 0.0f && isfinite(x)) ? x : 0.0f; }

__device__ __forceinline__ int fix_exp(float x) { return x != 0.0f ? ilogbf(x) : FIX_NONE; }

// x (counted) in fixed point relative to the column's exponent e
__device__ __forceinline__ long long fix_val(float x, int e)
{
    return x != 0.0f ? __float2ll_rn(scalbnf(x, FIX_SHIFT - e)) : 0ll;
}

__device__ __forceinline__ double fix_total(long long s, int e)
{
    return e == FIX_NONE ? 0.0 : ldexp((double)s, e - FIX_SHIFT);
}

}  // namespace msd
