// classes.cuh -- the size classes of the binned cell launches (variants 1-4)
// and the stream priorities of their launches: which cells run block-per-cell,
// warp-per-cell or packed, with which block size and capacity.
#pragma once
#include "common.cuh"

namespace msd {

// A class of cells by floe count, largest first: cells with more floes than
// the next class's bound and at most `hi`; `threads` per block; kind 0 block
// per cell, 1 warp per cell with the class bound as the warp capacity, 2
// several cells packed to a warp.
struct SizeClass {
    int hi, threads, kind;
};

// Variant 1 runs every class block-per-cell.  Variants 2-3 run cells above
// 256 floes block-per-cell in four classes (each class's shared memory is
// sized by its largest cell, so the split keeps most blocks small).  Variant
// 4's warp list kernel beats its block kernel up to 640 floes (measured on
// the 128 x 128 batched workload: 9.5 ms per coarse interval against 10.6 ms
// with block cells above 256 floes), so only larger cells run block-per-cell.
// Cells of at most 32 floes are packed.
constexpr SizeClass kClassesV1[4] = {{1 << 30, 256, 0}, {512, 256, 0}, {256, 128, 0}, {64, 64, 0}};
constexpr SizeClass kClassesV2[9] = {{1 << 30, 128, 0}, {640, 128, 0}, {512, 128, 0}, {384, 128, 0},
                                     {256, 128, 1},     {192, 128, 1}, {128, 128, 1}, {64, 128, 1},
                                     {32, 128, 2}};
constexpr SizeClass kClassesV4[9] = {{1 << 30, 128, 0}, {640, 128, 1}, {512, 128, 1}, {384, 128, 1},
                                     {256, 128, 1},     {192, 128, 1}, {128, 128, 1}, {64, 128, 1},
                                     {32, 128, 2}};

// Variant 5 keeps every cell of up to 1024 floes resident for a run of
// steps: cells of 513-1024 floes take a block with 4 floes per thread, of
// 257-512 floes 2 per thread, smaller cells share blocks a floe per thread
// (kind 3, the class bound / 256 floes per thread); larger cells run the
// block-per-cell list kernel step by step.
constexpr SizeClass kClassesV5[4] = {{1 << 30, 128, 0}, {1024, 256, 3}, {512, 256, 3}, {256, 256, 3}};

// The streams of the first kHighPriorityClasses size classes (the largest
// cells: few blocks, each holding much shared memory, and the longest
// launches) get the highest stream priority, so their blocks take SMs first
// as the other classes' blocks drain (measured on the 128 x 128 batched
// workload: 2-6 % less per interval than equal priorities or than priority
// for fewer classes; graded priorities were slower).
constexpr int kHighPriorityClasses = 4;
static_assert(sizeof(kClassesV2) / sizeof(SizeClass) <= MAXSEG && sizeof(kClassesV4) / sizeof(SizeClass) <= MAXSEG &&
                  sizeof(kClassesV5) / sizeof(SizeClass) <= MAXSEG,
              "more size classes than stream slots");

}  // namespace msd
