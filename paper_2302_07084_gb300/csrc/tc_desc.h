// Descriptor encodings of the tcgen05 tensor-core path (PTX ISA, sm_100a+),
// kept in a plain header so that a host program can check every field
// (tests/test_tc_desc.py).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define LNE_HD __host__ __device__
#else
#define LNE_HD
#endif

namespace lne {

// Instruction descriptor of tcgen05.mma .kind::tf32 with FP32 accumulation,
// both operands K-major, dense: bits 4-5 D format (1 = F32), 7-9 A format and
// 10-12 B format (2 = TF32), 13 / 14 negate A / B (0), 15 / 16 A / B major
// (0 = K-major), 17-22 N >> 3, 24-28 M >> 4; all other bits 0.
LNE_HD constexpr uint32_t tc_idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major operand stored in the 128-byte
// swizzle layout (rows of 128 bytes, 8-row atoms of 1024 bytes, as TMA writes
// with CU_TENSOR_MAP_SWIZZLE_128B): bits 0-13 start address >> 4, 16-29
// leading byte offset >> 4 (not used by this layout: 1), 32-45 stride byte
// offset >> 4 (1024 bytes from one 8-row group to the next), 46-48 the fixed
// value 0b001, 49-51 base offset (0: atoms start at 1024-byte boundaries),
// 52 leading-offset mode (0), 61-63 layout (2 = 128-byte swizzle).
LNE_HD constexpr uint64_t tc_sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

}  // namespace lne
