// Pencil FFTs held in registers (Sec. 3.3: Fourier transforms for the
// spatial derivatives).
//
// A pencil of length L = R * TH is owned by a group of TH consecutive lanes
// of one warp; lane t of the group holds R complex values.  Two layouts:
//
//   A layout: register r of lane t holds index  TH * r + t
//   B layout: register m * TH + k2 of lane j holds index (j + TH m) + R k2
//
// fft_ab maps A -> B and fft_ba maps B -> A; both compute the unnormalised
// sum  X[k] = sum_n x[n] exp(S * 2 pi i n k / L)  for the sign S given as a
// template argument.  Each is one radix-R (or radix-TH) DFT in registers, a
// twiddle multiply and one exchange through shared memory ordered with
// __syncwarp (a group never spans two warps).  Because the layouts alternate,
// a derivative ifft(i k fft(u)) needs no reordering between the transforms.
#pragma once

#include "rd_device.cuh"

namespace rd {

// Registers per lane for a pencil of length L (L = R * TH, TH | R, TH | 32).
__host__ __device__ constexpr int shape_r(int L) {
  return (L == 96) ? 24 : (L >= 128) ? 16 : (L >= 32 ? 8 : (L >= 8 ? 4 : 2));
}

template <int L>
struct Shape {
  static constexpr int R = shape_r(L);
  static constexpr int TH = L / R;       // lanes per pencil
  static constexpr int PAD = TH + 1;     // padded row of the exchange buffer
  static constexpr int GSTRIDE = R * PAD + ((R * PAD) % 16 == 0 ? 8 : 0);
  static constexpr int G = kThreads / TH;   // pencil groups per block
  static_assert(R >= TH, "stage B needs R >= TH");
  static_assert(32 % TH == 0, "a pencil group must sit inside one warp");
};

// cos(2 pi j / 16) for j in 0..15 (exact values of the 16th roots of unity).
template <typename T>
__device__ __forceinline__ T cos16(int j) {
  j &= 15;
  const T c1 = T(0.92387953251128675613), c2 = T(0.70710678118654752440),
          c3 = T(0.38268343236508977173);
  switch (j) {
    case 0: return T(1);
    case 1: return c1;
    case 2: return c2;
    case 3: return c3;
    case 4: return T(0);
    case 5: return -c3;
    case 6: return -c2;
    case 7: return -c1;
    case 8: return T(-1);
    case 9: return -c1;
    case 10: return -c2;
    case 11: return -c3;
    case 12: return T(0);
    case 13: return c3;
    case 14: return c2;
    default: return c1;
  }
}

// cos(2 pi j / 24) for j in 0..23 (exact values of the 24th roots of unity).
template <typename T>
__device__ __forceinline__ T cos24(int j) {
  j = ((j % 24) + 24) % 24;
  const T c1 = T(0.96592582628906828675), c2 = T(0.86602540378443864676), c3 = T(0.70710678118654752440),
          c4 = T(0.5), c5 = T(0.25881904510252076235);
  const int q = (j > 12) ? 24 - j : j;   // cos is even
  switch (q) {
    case 0: return T(1);
    case 1: return c1;
    case 2: return c2;
    case 3: return c3;
    case 4: return c4;
    case 5: return c5;
    case 6: return T(0);
    case 7: return -c5;
    case 8: return -c4;
    case 9: return -c3;
    case 10: return -c2;
    case 11: return -c1;
    default: return T(-1);
  }
}

// x * exp(S * 2 pi i k / M) for a compile-time-resolvable k; M divides 16
// or 24.
template <typename T, int M, int S>
__device__ __forceinline__ cpx<T> twk(int k, cpx<T> x) {
  if constexpr (16 % M == 0) {
    const int j = (k * 16 / M) & 15;
    if (j == 0) return x;
    if (j == 4) return {-T(S) * x.y, T(S) * x.x};
    if (j == 8) return {-x.x, -x.y};
    if (j == 12) return {T(S) * x.y, -T(S) * x.x};
    const T c = cos16<T>(j), s = T(S) * cos16<T>(j - 4);
    return cmul(x, c, s);
  } else {
    static_assert(24 % M == 0, "twiddle denominator must divide 16 or 24");
    const int j = (k * 24 / M) % 24;
    if (j == 0) return x;
    if (j == 6) return {-T(S) * x.y, T(S) * x.x};
    if (j == 12) return {-x.x, -x.y};
    if (j == 18) return {T(S) * x.y, -T(S) * x.x};
    const T c = cos24<T>(j), s = T(S) * cos24<T>(j - 6);
    return cmul(x, c, s);
  }
}

// In-register DFT of M points, natural order in and out, sign S.
template <typename T, int M, int S>
struct Dft {
  __device__ __forceinline__ static void run(cpx<T>* x) {
    cpx<T> e[M / 2], o[M / 2];
#pragma unroll
    for (int i = 0; i < M / 2; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    Dft<T, M / 2, S>::run(e);
    Dft<T, M / 2, S>::run(o);
#pragma unroll
    for (int k = 0; k < M / 2; ++k) {
      cpx<T> t = twk<T, M, S>(k, o[k]);
      x[k] = e[k] + t;
      x[k + M / 2] = e[k] - t;
    }
  }
};
template <typename T, int S>
struct Dft<T, 1, S> {
  __device__ __forceinline__ static void run(cpx<T>*) {}
};
// 3-point DFT: X_k = sum_n x_n w^{nk}, w = exp(S 2 pi i / 3) = (-1/2, S sqrt(3)/2).
template <typename T, int S>
struct Dft<T, 3, S> {
  __device__ __forceinline__ static void run(cpx<T>* x) {
    const T h = T(0.86602540378443864676) * T(S);
    const cpx<T> a = x[0], b = x[1], c = x[2];
    const cpx<T> sbc = b + c, dbc = b - c;
    const cpx<T> m = {a.x - T(0.5) * sbc.x, a.y - T(0.5) * sbc.y};
    // w b + w^2 c = -1/2 (b + c) + i S sqrt(3)/2 (b - c)
    const cpx<T> rot = {-h * dbc.y, h * dbc.x};
    x[0] = a + sbc;
    x[1] = m + rot;
    x[2] = m - rot;
  }
};
template <typename T, int S>
struct Dft<T, 2, S> {
  __device__ __forceinline__ static void run(cpx<T>* x) {
    cpx<T> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  }
};

// Read-only cached load of one complex table entry.
template <typename T>
__device__ __forceinline__ cpx<T> ldtw(const cpx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
  } else {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
  }
}

// Where a transform reads its twiddles from (template argument TW):
//   kTwLdg    global memory through the read-only path (__ldg);
//   kTwShared a shared-memory copy of the table, volatile loads;
//   kTwGlobal global memory through L1, volatile loads.
// The volatile forms make the compiler re-read a twiddle at each use instead
// of keeping every twiddle of a persistent loop live in registers (230
// registers instead of 96).  Kernels whose occupancy is limited by shared
// memory use kTwGlobal and keep the 4 KB table out of shared memory.
constexpr int kTwLdg = 0, kTwShared = 1, kTwGlobal = 2;

template <typename T>
__device__ __forceinline__ cpx<T> ldtw_shared(const cpx<T>* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  cpx<T> v;
  if constexpr (sizeof(T) == 4) {
    asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  } else {
    asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
  }
  return v;
}

template <typename T>
__device__ __forceinline__ cpx<T> ldtw_global(const cpx<T>* p) {
  cpx<T> v;
  if constexpr (sizeof(T) == 4) {
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  } else {
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  }
  return v;
}

template <int TW, typename T>
__device__ __forceinline__ cpx<T> ldtw_any(const cpx<T>* p) {
  if constexpr (TW == kTwShared) return ldtw_shared(p);
  else if constexpr (TW == kTwGlobal) return ldtw_global(p);
  else return ldtw(p);
}

// Twiddle tables (host-computed in FP64, stored in global memory per L):
//   twA[k1 * TH + t]          = exp(-2 pi i t k1 / L)
//   twB[(m * TH + n2) * TH + j] = exp(+2 pi i n2 (j + TH m) / L)
template <typename T, int L, int S, int SH = kTwLdg>
__device__ __forceinline__ void fft_ab(cpx<T>* v, cpx<T>* sm, int t, const cpx<T>* __restrict__ twA) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, PAD = Sh::PAD;
  Dft<T, R, S>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) {
    cpx<T> w = ldtw_any<SH>(&twA[k1 * TH + t]);
    v[k1] = cmul(v[k1], w.x, S < 0 ? w.y : -w.y);
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) sm[k1 * PAD + t] = v[k1];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < R / TH; ++m)
#pragma unroll
    for (int n2 = 0; n2 < TH; ++n2) v[m * TH + n2] = sm[(t + TH * m) * PAD + n2];
#pragma unroll
  for (int m = 0; m < R / TH; ++m) Dft<T, TH, S>::run(v + m * TH);
}

template <typename T, int L, int S, int SH = kTwLdg>
__device__ __forceinline__ void fft_ba(cpx<T>* u, cpx<T>* sm, int j, const cpx<T>* __restrict__ twB) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, PAD = Sh::PAD;
#pragma unroll
  for (int m = 0; m < R / TH; ++m) Dft<T, TH, S>::run(u + m * TH);
#pragma unroll
  for (int m = 0; m < R / TH; ++m)
#pragma unroll
    for (int n2 = 0; n2 < TH; ++n2) {
      if (n2 == 0) continue;
      cpx<T> w = ldtw_any<SH>(&twB[(m * TH + n2) * TH + j]);
      u[m * TH + n2] = cmul(u[m * TH + n2], w.x, S > 0 ? w.y : -w.y);
    }
  __syncwarp();
#pragma unroll
  for (int m = 0; m < R / TH; ++m)
#pragma unroll
    for (int n2 = 0; n2 < TH; ++n2) sm[(j + TH * m) * PAD + n2] = u[m * TH + n2];
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) u[k1] = sm[k1 * PAD + j];
  Dft<T, R, S>::run(u);
}

// Complex conjugate of R register values: an inverse transform is the
// forward one between two conjugations (exact: only signs change).
template <typename T, int R>
__device__ __forceinline__ void conj_all(cpx<T>* v) {
#pragma unroll
  for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
}

// Index held by register r of lane t in each layout.
template <int L>
__device__ __forceinline__ int idx_a(int r, int t) { return Shape<L>::TH * r + t; }
template <int L>
__device__ __forceinline__ int idx_b(int r, int j) {
  constexpr int R = Shape<L>::R, TH = Shape<L>::TH;
  return (j + TH * (r / TH)) + R * (r % TH);
}

// Signed wavenumber of index k with the Nyquist index mapped to zero (the
// first-derivative symbol i k~ vanishes there).
template <int L>
__device__ __forceinline__ int kwave(int k) {
  return (k < L / 2) ? k : (k == L / 2 ? 0 : k - L);
}

// Register that holds index (L - k) mod L, for lanes t > 0 (on lane TH - t)
// and for lane 0 (on itself).
template <int L>
__device__ __forceinline__ constexpr int mirror_b_other(int r) {
  constexpr int R = Shape<L>::R, TH = Shape<L>::TH;
  return (R / TH - 1 - r / TH) * TH + (TH - 1 - r % TH);
}
template <int L>
__device__ __forceinline__ constexpr int mirror_b_zero(int r) {
  constexpr int R = Shape<L>::R, TH = Shape<L>::TH;
  return (r / TH == 0) ? ((TH - r % TH) % TH) : ((R / TH - r / TH) * TH + (TH - 1 - r % TH));
}
template <int L>
__device__ __forceinline__ constexpr int mirror_a_other(int r) { return Shape<L>::R - 1 - r; }
template <int L>
__device__ __forceinline__ constexpr int mirror_a_zero(int r) { return (Shape<L>::R - r) % Shape<L>::R; }

// mir[r] = the value at index (L - k) mod L of the pencil, k the index held
// by register r (layout B or A); fetched from the mirror lane of the group.
template <typename T, int L, bool LAYOUT_B>
__device__ __forceinline__ void mirror_fetch(const cpx<T>* v, cpx<T>* mir, int t) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH;
  const int lane = threadIdx.x & 31;
  const int src = (lane & ~(TH - 1)) | ((TH - t) & (TH - 1));
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int ro = LAYOUT_B ? mirror_b_other<L>(r) : mirror_a_other<L>(r);
    const int rz = LAYOUT_B ? mirror_b_zero<L>(r) : mirror_a_zero<L>(r);
    T mx = __shfl_sync(0xffffffffu, v[ro].x, src);
    T my = __shfl_sync(0xffffffffu, v[ro].y, src);
    mir[r].x = (t == 0) ? v[rz].x : mx;
    mir[r].y = (t == 0) ? v[rz].y : my;
  }
}

// Given Z = F(a + i b) (forward sign) in layout B (or A), replace every
// register by (H a, H b): the discrete Hartley transforms
// H x[k] = sum_n x[n] (cos + sin)(2 pi n k / L) of the two real sequences.
// H a[k] = (Re Z_k + Re Z_-k - Im Z_k + Im Z_-k) / 2
// H b[k] = (Re Z_k - Re Z_-k + Im Z_k + Im Z_-k) / 2
template <typename T, int L, bool LAYOUT_B>
__device__ __forceinline__ void hartley_combine(cpx<T>* v, int t) {
  constexpr int R = Shape<L>::R;
  cpx<T> mir[R];
  mirror_fetch<T, L, LAYOUT_B>(v, mir, t);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    cpx<T> z = v[r], m = mir[r];
    v[r].x = T(0.5) * ((z.x + m.x) - (z.y - m.y));
    v[r].y = T(0.5) * ((z.x - m.x) + (z.y + m.y));
  }
}

}  // namespace rd
