// Kernels of the registration sub-problem (Sec. 2.1 Eq. reg:fwd, reg:adj,
// reg:inv; Sec. 2.2 Eq. objective_reg; Sec. 3.2 and 3.3 numerics):
// semi-Lagrangian transport with tricubic Lagrange interpolation at Heun
// characteristic feet, spectral first and second derivatives along one axis,
// the axis-0 pass of a constant-coefficient spectral solve, and the
// pointwise pieces of the objective and the adjoint final conditions.
#pragma once

#include "rd_fft.cuh"
#include "rd_passes.cuh"

namespace rd {
namespace reg {

// Cubic Lagrange weights of the nodes -1, 0, 1, 2 at offset f in [0, 1).
template <typename T>
__device__ __forceinline__ void lag4(T f, T* w) {
  const T fm1 = f - T(1), fm2 = f - T(2), fp1 = f + T(1);
  w[0] = -f * fm1 * fm2 * T(1.0 / 6.0);
  w[1] = fp1 * fm1 * fm2 * T(0.5);
  w[2] = -fp1 * f * fm2 * T(0.5);
  w[3] = fp1 * f * fm1 * T(1.0 / 6.0);
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// K separate fields interpolated at the point (X0, X1, X2) in index units,
// periodic: the same tricubic Lagrange stencil as interp4, one scalar load
// per field and neighbour (used where packing would waste loaded bytes).
template <typename T, int K>
__device__ __forceinline__ void interp_fields(const T* const* u, const Geom& g, T X0, T X1, T X2, T* out) {
  const T f0 = floor(X0), f1 = floor(X1), f2 = floor(X2);
  T w0[4], w1[4], w2[4];
  lag4(X0 - f0, w0);
  lag4(X1 - f1, w1);
  lag4(X2 - f2, w2);
  const int b0 = int(f0) - 1, b1 = int(f1) - 1, b2 = int(f2) - 1;
  int i2[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) i2[o] = wrap(b2 + o, g.n[2]);
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = T(0);
#pragma unroll
  for (int o0 = 0; o0 < 4; ++o0) {
    const int i0 = wrap(b0 + o0, g.n[0]);
#pragma unroll
    for (int o1 = 0; o1 < 4; ++o1) {
      const long long row = ((long long)i0 * g.n[1] + wrap(b1 + o1, g.n[1])) * g.n[2];
      const T w01 = w0[o0] * w1[o1];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T* p = u[k] + row;
        // read-only path: the gathered fields are never written by this kernel
        const T acc = w2[0] * __ldg(p + i2[0]) + w2[1] * __ldg(p + i2[1]) + w2[2] * __ldg(p + i2[2]) +
                      w2[3] * __ldg(p + i2[3]);
        out[k] += w01 * acc;
      }
    }
  }
}

// Four fields of one grid point side by side (array of structures), so that
// the 64-point stencil of an interpolation loads each neighbour once with a
// vector load instead of once per field.
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

template <typename T>
__device__ __forceinline__ V4<T> ldv4(const V4<T>* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {a.x, a.y, b.x, b.y};
  }
}

// out[i] = (a[i], b[i], c[i], d ? d[i] : 0)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pack4(const T* __restrict__ a, const T* __restrict__ b,
                                                    const T* __restrict__ c, const T* __restrict__ d,
                                                    V4<T>* __restrict__ out, long long nn) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads)
    out[i] = {a[i], b[i], c[i], d ? d[i] : T(0)};
}

// Periodic tricubic Lagrange interpolation (nodes -1..2 per axis, weights
// lag4) at the point (X0, X1, X2) in index units, for NP packed arrays of
// four fields each: out[4 p + j] is component j of array p there.  The
// weights are applied axis by axis (rows along axis 2 first).
template <typename T, int NP>
__device__ __forceinline__ void interp4(const V4<T>* const* u, const Geom& g, T X0, T X1, T X2, T* out) {
  const T f0 = floor(X0), f1 = floor(X1), f2 = floor(X2);
  T w0[4], w1[4], w2[4];
  lag4(X0 - f0, w0);
  lag4(X1 - f1, w1);
  lag4(X2 - f2, w2);
  const int b0 = int(f0) - 1, b1 = int(f1) - 1, b2 = int(f2) - 1;
  int i2[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) i2[o] = wrap(b2 + o, g.n[2]);
#pragma unroll
  for (int k = 0; k < 4 * NP; ++k) out[k] = T(0);
#pragma unroll
  for (int o0 = 0; o0 < 4; ++o0) {
    const int i0 = wrap(b0 + o0, g.n[0]);
#pragma unroll
    for (int o1 = 0; o1 < 4; ++o1) {
      const long long row = ((long long)i0 * g.n[1] + wrap(b1 + o1, g.n[1])) * g.n[2];
      const T w01 = w0[o0] * w1[o1];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const V4<T>* p = u[q] + row;
        V4<T> acc = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int o2 = 0; o2 < 4; ++o2) {
          const V4<T> e = ldv4(p + i2[o2]);
          acc.x += w2[o2] * e.x;
          acc.y += w2[o2] * e.y;
          acc.z += w2[o2] * e.z;
          acc.w += w2[o2] * e.w;
        }
        out[4 * q + 0] += w01 * acc.x;
        out[4 * q + 1] += w01 * acc.y;
        out[4 * q + 2] += w01 * acc.z;
        out[4 * q + 3] += w01 * acc.w;
      }
    }
  }
}

__device__ __forceinline__ void coords(const Geom& g, long long i, int& i0, int& i1, int& i2) {
  i2 = int(i % g.n[2]);
  const long long r = i / g.n[2];
  i1 = int(r % g.n[1]);
  i0 = int(r / g.n[1]);
}

// Characteristic foot as a displacement in index units:
// d = sign dt/2 (v(x) + v(x + sign dt v(x))) / h  (Heun's rule, stationary v).
template <typename T>
struct FeetArgs {
  const T* v[3];
  const V4<T>* vp;   // (v0, v1, v2, 0) packed for the interpolation
  T* d[3];
  Geom g;
  T cdt[3];   // sign * dt / h_a
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_feet(FeetArgs<T> a) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.g.nn; i += (long long)gridDim.x * kThreads) {
    int i0, i1, i2;
    coords(a.g, i, i0, i1, i2);
    const T v0 = a.v[0][i], v1 = a.v[1][i], v2 = a.v[2][i];
    T vy[4];
    interp4<T, 1>(&a.vp, a.g, T(i0) + a.cdt[0] * v0, T(i1) + a.cdt[1] * v1, T(i2) + a.cdt[2] * v2, vy);
    a.d[0][i] = T(0.5) * a.cdt[0] * (v0 + vy[0]);
    a.d[1][i] = T(0.5) * a.cdt[1] * (v1 + vy[1]);
    a.d[2][i] = T(0.5) * a.cdt[2] * (v2 + vy[2]);
  }
}

enum InterpMode {
  kIpPlain = 0,   // out_k = u_k(X)
  kIpAdj = 1,     // out_k = l_k(X) + dt/2 (l_k(X) D(X) + (l_k(X) + dt l_k(X) D(X)) D(x))
  kIpInc = 2      // out_k = u_k(X) - dt/2 (s_k(X) + s1_k(x))
};

template <typename T>
struct InterpArgs {
  const T* d[3];
  const T* u[3];
  const T* s[3];    // kIpInc: source at the previous level
  const T* s1[3];   // kIpInc: source at the new level
  const T* D;       // kIpAdj: div v
  const V4<T>* pk[1];   // plain/adjoint: the gathered fields packed, (u0, u1, u2, D or 0)
  T* out[3];
  Geom g;
  T dt;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_interp(InterpArgs<T> a) {
  // plain and adjoint: the gathered fields packed by k_pack4, (u, 0) and
  // (l, D), one vector load per neighbour; incremental: six separate fields
  // (u and s), where packing would load two pad values per neighbour
  const T* src6[6] = {a.u[0], a.u[1], a.u[2], a.s[0], a.s[1], a.s[2]};
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.g.nn; i += (long long)gridDim.x * kThreads) {
    int i0, i1, i2;
    coords(a.g, i, i0, i1, i2);
    const T X0 = T(i0) + a.d[0][i], X1 = T(i1) + a.d[1][i], X2 = T(i2) + a.d[2][i];
    T r[6];
    if constexpr (MODE == kIpInc) {
      interp_fields<T, 6>(src6, a.g, X0, X1, X2, r);
    } else {
      interp4<T, 1>(a.pk, a.g, X0, X1, X2, r);
    }
    if constexpr (MODE == kIpPlain) {
#pragma unroll
      for (int k = 0; k < 3; ++k) a.out[k][i] = r[k];
    } else if constexpr (MODE == kIpAdj) {
      const T DX = r[3], Dx = a.D[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T pred = r[k] + a.dt * r[k] * DX;
        a.out[k][i] = r[k] + T(0.5) * a.dt * (r[k] * DX + pred * Dx);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) a.out[k][i] = r[k] - T(0.5) * a.dt * (r[3 + k] + a.s1[k][i]);
    }
  }
}

// ------------------------------------------------ spectral derivative pass
// d = (i k~)^order applied along `axis` (Nyquist symbol zeroed), scaled by c:
//   kDerSet: out = c d u;  kDerAdd: out += c d u;  kDerMulAdd: out += c w d u.
enum DerMode { kDerSet = 0, kDerAdd = 1, kDerMulAdd = 2 };

template <typename T>
struct DerivArgs {
  const T* u;
  const T* w;
  T* out;
  double c;
  int axis;
  int order;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
};

template <typename T, int L, bool CONTIG, int MODE>
__global__ void __launch_bounds__(kThreads) k_deriv(DerivArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const T c = T(a.c / double(L));
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<CONTIG>(a.g, a.axis, act ? pair : 0, b0, b1, st);
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[r] = act ? ld2<T, CONTIG>(a.u, b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
    fft_ab<T, L, -1>(v, sm, t, a.twA);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = kwave<L>(idx_b<L>(r, t));
      if (a.order == 1) {
        v[r] = times_ik(v[r], k);
      } else {
        const T kk = -T(k) * T(k);
        v[r] = {kk * v[r].x, kk * v[r].y};
      }
    }
    fft_ba<T, L, +1>(v, sm, t, a.twB);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long off = (long long)idx_a<L>(r, t) * st;
        cpx<T> o = {c * v[r].x, c * v[r].y};
        if constexpr (MODE == kDerMulAdd) {
          const cpx<T> w = ld2<T, CONTIG>(a.w, b0, b1, off);
          o = {o.x * w.x, o.y * w.y};
        }
        if constexpr (MODE != kDerSet) {
          const cpx<T> p = ld2<T, CONTIG>(a.out, b0, b1, off);
          o = {o.x + p.x, o.y + p.y};
        }
        st2<T, CONTIG>(a.out, b0, b1, off, o);
      }
    }
  }
}

// Three first derivatives along `axis` in one pass (three transforms per
// pencil pair, one read-modify-write of the outputs):
//   kD3Body: out[0] += c sum_k w[k] d u[k]      (body force sum_i l_i d_a m_i)
//   kD3Src:  out[k] += c w[0] d u[k], k = 0..2   (source grad(m_k) . v~, axis term)
enum Deriv3Mode { kD3Body = 0, kD3Src = 1 };

template <typename T>
struct Deriv3Args {
  const T* u[3];
  const T* w[3];
  T* out[3];
  double c;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
};

template <typename T, int L, bool CONTIG, int MODE>
__global__ void __launch_bounds__(kThreads) k_deriv3(const __grid_constant__ Deriv3Args<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const T c = T(a.c / double(L));
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<CONTIG>(a.g, a.axis, act ? pair : 0, b0, b1, st);
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      cpx<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[r] = act ? ld2<T, CONTIG>(a.u[k], b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
      fft_ab<T, L, -1>(v, sm, t, a.twA);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
      fft_ba<T, L, +1>(v, sm, t, a.twB);
      if (act) {
        const T* w = a.w[MODE == kD3Body ? k : 0];
        T* out = a.out[MODE == kD3Body ? 0 : k];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const long long off = (long long)idx_a<L>(r, t) * st;
          const cpx<T> wv = ld2<T, CONTIG>(w, b0, b1, off);
          const cpx<T> p = ld2<T, CONTIG>(out, b0, b1, off);
          st2<T, CONTIG>(out, b0, b1, off, {p.x + c * wv.x * v[r].x, p.y + c * wv.y * v[r].y});
        }
      }
    }
  }
}

// ------------------------------------ spectral solve: the axis-0 symbol pass
// Between Hartley passes along axes 2 and 1 (before and after), applies
// F_0^-1 S F_0 along axis 0 with S(k) = inn / (a1 |k~|^2) where |k~|^2 > 0
// and inn * z0 where it vanishes (|k~|^2 over all three axes; the symbol is
// real and even, so this equals H_0 S H_0).
template <typename T>
struct SolveArgs {
  const T* in;
  T* out;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  double a1;
  double z0;
  double inn;
};

template <typename T>
__device__ __forceinline__ T solve_symbol(T kk, T a1, T z0, T inn) {
  return kk > T(0) ? inn / (a1 * kk) : inn * z0;
}

template <typename T, int L>
__global__ void __launch_bounds__(kThreads) k_solve0(SolveArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const T a1 = T(a.a1), z0 = T(a.z0), inn = T(a.inn);
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<false>(a.g, 0, act ? pair : 0, b0, b1, st);
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[r] = act ? ld2<T, false>(a.in, b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
    fft_ab<T, L, -1>(v, sm, t, a.twA);
    // pencils (i1, i2) and (i1, i2 + 1)
    const long long P = 2 * (act ? pair : 0);
    const int i1 = int(P / a.g.n[2]), i2 = int(P % a.g.n[2]);
    const int k1 = kwave_rt(i1, a.g.n[1]), k2a = kwave_rt(i2, a.g.n[2]), k2b = kwave_rt(i2 + 1, a.g.n[2]);
    const T base_a = T(k1 * k1 + k2a * k2a), base_b = T(k1 * k1 + k2b * k2b);
    cpx<T> mir[R];
    mirror_fetch<T, L, true>(v, mir, t);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k0 = kwave<L>(idx_b<L>(r, t));
      const T kk = T(k0 * k0);
      const T sa = solve_symbol(base_a + kk, a1, z0, inn), sb = solve_symbol(base_b + kk, a1, z0, inn);
      const cpx<T> z = v[r], m = mir[r];
      const T hp = T(0.5) * (sa + sb), hm = T(0.5) * (sa - sb);
      v[r].x = hp * z.x + hm * m.x;
      v[r].y = hp * z.y - hm * m.y;
    }
    fft_ba<T, L, +1>(v, sm, t, a.twB);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) st2<T, false>(a.out, b0, b1, (long long)idx_a<L>(r, t) * st, v[r]);
    }
  }
}

// ------------------------------------------------------ pointwise pieces
// kFinalState: r_i = (1 - c) m_i - m_P,i; sum 1/2 r_i^2 + q_i m_i into the
// partials; l_i = -((1 - c) r_i + q_i).   kFinalInc: l_i = -(1 - c)^2 m_i.
enum FinalMode { kFinalState = 0, kFinalInc = 1 };

template <typename T>
struct FinalArgs {
  const T* m[3];
  const T* mp[3];
  const T* c;
  const T* q[3];   // may be null
  T* lam[3];
  double* part;
  long long nn;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_final(FinalArgs<T> a) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.nn; i += (long long)gridDim.x * kThreads) {
    const T w = T(1) - a.c[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if constexpr (MODE == kFinalState) {
        const T r = w * a.m[k][i] - a.mp[k][i];
        const T qk = a.q[k] ? a.q[k][i] : T(0);
        acc += 0.5 * double(r) * double(r) + double(qk) * double(a.m[k][i]);
        a.lam[k][i] = -(w * r + qk);
      } else {
        a.lam[k][i] = -(w * w) * a.m[k][i];
      }
    }
  }
  if constexpr (MODE == kFinalState) {
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.part[blockIdx.x] = red[0];
  }
}

// Deterministic FP64 dot product of two 3-component fields: per-block
// partials in a fixed order, then one block sums them in a fixed order.
template <typename T>
struct DotArgs {
  const T* x[3];
  const T* y[3];
  double* part;
  long long nn;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot3(DotArgs<T> a) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.nn; i += (long long)gridDim.x * kThreads)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc += double(a.x[k][i]) * double(a.y[k][i]);
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads) k_sum_parts(const double* part, int n, double* out) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace reg
}  // namespace rd
