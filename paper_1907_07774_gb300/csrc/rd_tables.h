// Host-side helpers shared by the engines: twiddle tables of the pencil FFT
// (computed in FP64) and pointer classification.
#pragma once

#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "rd_fft.cuh"

namespace rd {

constexpr double kTwoPiHost = 6.283185307179586476925286766559;
constexpr int kNumL = 7;   // pencil lengths 8, 16, 32, 64, 128, 256 and 96

inline int lidx(int L) {
  if (L == 96) return 6;
  int i = 0;
  while ((8 << i) < L) ++i;
  return i;
}

inline int slot_length(int i) { return i == 6 ? 96 : (8 << i); }

// Tables of the two stages of fft_ab / fft_ba for pencil length L:
//   ta[k1 * TH + t]          = exp(-2 pi i t k1 / L)
//   tb[(m * TH + n2) * TH + j] = exp(+2 pi i n2 (j + TH m) / L)
template <typename T>
void build_twiddles(int L, std::vector<cpx<T>>& ta, std::vector<cpx<T>>& tb) {
  const int R = shape_r(L);
  const int TH = L / R;
  ta.assign(L, cpx<T>{T(0), T(0)});
  tb.assign(L, cpx<T>{T(0), T(0)});
  for (int k1 = 0; k1 < R; ++k1)
    for (int t = 0; t < TH; ++t) {
      const double th = kTwoPiHost * double((long long)t * k1 % L) / L;
      ta[k1 * TH + t] = {T(std::cos(th)), T(-std::sin(th))};
    }
  for (int m = 0; m < R / TH; ++m)
    for (int n2 = 0; n2 < TH; ++n2)
      for (int j = 0; j < TH; ++j) {
        const int k1 = j + TH * m;
        const double th = kTwoPiHost * double((long long)n2 * k1 % L) / L;
        tb[(m * TH + n2) * TH + j] = {T(std::cos(th)), T(std::sin(th))};
      }
}

inline bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace rd
