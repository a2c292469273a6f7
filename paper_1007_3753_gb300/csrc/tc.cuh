// TMA tensor maps of the tensor-core sweeps (host side).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace l1 {
namespace tc {

// Tiled 2-D tensor map over `rows` rows of `inner` BF16 elements, row pitch
// pitch_bytes; box = box_inner elements (64: 128 bytes, 128-byte swizzle; 32:
// 64 bytes, 64-byte swizzle) x box_rows.
// Returns L1_OK, L1_ERR_INVALID_ARG (misaligned base or pitch, another box
// width) or L1_ERR_CUDA.
int make_map_bf16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
                  uint32_t box_inner, uint32_t box_rows);

}  // namespace tc
}  // namespace l1
