// Host helpers for the tcgen05 kernels: TMA descriptors and launch set-up.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace crl {
namespace tc {

// 2-D BF16 tensor map over a row-major [rows][inner] array with row stride
// `row_stride_elems` (a multiple of 8), box {64, box_rows}, 128-byte swizzle,
// zero fill outside the array.  Returns false (and sets *err) on failure.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint64_t row_stride_elems,
                    uint32_t box_rows, const char** err);

}  // namespace tc
}  // namespace crl
