// Host helper for TMA tensor maps (the driver entry point is resolved once at
// run time, so the library links against the CUDA runtime only).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace nys {

// 2-D FP32 tensor map over a row-major [rows x cols] array with row stride ld
// (elements, ld * 4 a multiple of 16, base 16-byte aligned); box =
// [box_rows x box_cols] with box_cols * 4 <= 128, 128-byte swizzle.  Returns
// false when the driver entry point is missing or rejects the map.
bool tmap_f32_2d(CUtensorMap* tm, const float* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_rows, int box_cols);
// The same for FP16 elements (ld * 2 a multiple of 16, box_cols * 2 <= 128).
bool tmap_f16_2d(CUtensorMap* tm, const void* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_rows, int box_cols);

}  // namespace nys
