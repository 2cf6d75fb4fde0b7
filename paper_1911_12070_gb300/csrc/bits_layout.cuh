// bits_layout.cuh -- layout shared by the bit-sliced sweep (sweep_bits.cu),
// which writes one 16-byte record per lane and plane with faces, and the
// expand pass (expand_bits.cu), which reads them: bands of 16 owned rows (one
// bit each in the L and H words of a record) plus a halo row, warps of 31
// owned columns (lane 31 is the next warp's first column).
#pragma once

#include <stdint.h>

namespace qtv {
namespace bits {
constexpr int BR = 16;            // owned rows per band
constexpr int BRH = BR + 1;       // plus the halo row
constexpr int BL = 31;            // owned columns per warp
constexpr uint32_t kRows16 = 0xFFFFu;
}  // namespace bits
}  // namespace qtv
