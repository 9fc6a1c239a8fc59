// FFT length limits shared by the host length choice and the device kernels.
#pragma once

namespace mm {

// Longest complex64 line the device FFT keeps in registers: 32 RR points with
// RR <= kRegFftMax (one warp per line, RR points per lane).
constexpr int kRegFftMax = 12;

}  // namespace mm
