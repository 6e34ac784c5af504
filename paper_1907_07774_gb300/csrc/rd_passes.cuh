// Axis passes and pointwise kernels of the reaction-diffusion solve.
//
// Every axis pass walks the pencils of one grid axis two at a time: the two
// real pencils (adjacent rows for the contiguous axis 2, adjacent columns
// for the strided axes 0 and 1) are packed as the real and imaginary parts
// of one complex pencil.  All operators applied along a pencil are real, so
// the packing is exact.
//
// Operator (Sec. 3.3, pseudo-spectral): A u = div(kappa grad u) =
// sum_a d_a(kappa d_a u), and d_a = F_a^-1 (i k~_a) F_a only involves the 1D
// transform along axis a (the other axes' transforms cancel), so A is
// applied as three axis passes, each holding whole pencils of u and kappa.
//
// Preconditioner: M^-1 = F^-1 diag(1 / (1 + s kbar |k~|^2)) F.  Its symbol is
// real and even in every wavenumber component, so it is also diagonalised by
// the separable Hartley transform H = H_0 H_1 H_2 (H_a H_a = n_a I); the
// preconditioner is applied as H_2, H_1, (H_0 S H_0), H_1, H_2 on real data.
#pragma once

#include "rd_fft.cuh"

namespace rd {

// ------------------------------------------------------------------ access
template <bool CONTIG>
__device__ __forceinline__ void pair_addr(const Geom& g, int axis, long long pair, long long& b0,
                                          long long& b1, long long& st) {
  const long long P = 2 * pair;
  if (CONTIG) {  // axis 2
    b0 = P * g.n[2];
    b1 = b0 + g.n[2];
    st = 1;
  } else if (axis == 1) {
    const long long i0 = P / g.n[2], i2 = P % g.n[2];
    b0 = i0 * (long long)g.n[1] * g.n[2] + i2;
    b1 = b0 + 1;
    st = g.n[2];
  } else {  // axis 0
    b0 = P;
    b1 = P + 1;
    st = (long long)g.n[1] * g.n[2];
  }
}

template <typename T, bool CONTIG>
__device__ __forceinline__ cpx<T> ld2(const T* f, long long b0, long long b1, long long off) {
  if (CONTIG) {
    return {f[b0 + off], f[b1 + off]};
  } else {
    if constexpr (sizeof(T) == 4) {
      float2 v = *reinterpret_cast<const float2*>(f + b0 + off);
      return {T(v.x), T(v.y)};
    } else {
      double2 v = *reinterpret_cast<const double2*>(f + b0 + off);
      return {T(v.x), T(v.y)};
    }
  }
}

template <typename T, bool CONTIG>
__device__ __forceinline__ void st2(T* f, long long b0, long long b1, long long off, cpx<T> v) {
  if (CONTIG) {
    f[b0 + off] = v.x;
    f[b1 + off] = v.y;
  } else {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float2*>(f + b0 + off) = make_float2(v.x, v.y);
    } else {
      *reinterpret_cast<double2*>(f + b0 + off) = make_double2(v.x, v.y);
    }
  }
}

template <int L>
__device__ __forceinline__ int pos_of(bool layout_b, int r, int t) {
  return layout_b ? idx_b<L>(r, t) : idx_a<L>(r, t);
}

template <typename T>
__device__ __forceinline__ cpx<T> times_ik(cpx<T> v, int k) {
  return {-T(k) * v.y, T(k) * v.x};
}

// 1/x for x >= 1 in the working precision.  FP32: the approximate PTX
// reciprocal (a relative error of about 2^-23; it only enters the
// preconditioner symbol, which changes how fast PCG converges, not what it
// converges to).
// FP64: an FP32 reciprocal refined by two Newton-Raphson steps
// r <- r (2 - x r) (each step squares the relative error, 2^-24 -> 2^-96),
// which avoids the much slower FP64 division on this part.
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) {
  double r = double(1.0f / float(x));
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
}

// Preconditioner symbol along axis 0 applied in the Fourier domain.  With
// Z = F(a + i b) (forward sign, layout B) for two real pencils a, b whose
// symbols S'_a(k), S'_b(k) are real and even in k, H S' H x = F^-1 (S' F x)
// (unnormalised inverse; the odd sine parts cancel), so
//   W_k = S'_a A_k + i S'_b B_k = (S'_a + S'_b)/2 Z_k + (S'_a - S'_b)/2 conj(Z_-k)
// with A_k = (Z_k + conj Z_-k)/2, B_k = (Z_k - conj Z_-k)/(2i); and since
// sum_k S'(k) (H a)_k^2 = sum_k S'(k) |A_k|^2 for an even S', the returned
// sum_k S'_a |A_k|^2 + S'_b |B_k|^2 is the Hartley-domain r.z term.
template <typename T, int L>
__device__ __forceinline__ T sym_apply(cpx<T>* v, int t, T base_a, T base_b, T symcT, T innT) {
  constexpr int R = Shape<L>::R;
  cpx<T> mir[R];
  mirror_fetch<T, L, true>(v, mir, t);
  T loc = T(0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k0 = kwave<L>(idx_b<L>(r, t));
    const T kk = T(k0 * k0);
    const T sa = innT * recip(T(1) + symcT * (base_a + kk));
    const T sb = innT * recip(T(1) + symcT * (base_b + kk));
    const cpx<T> z = v[r], m = mir[r];
    const T ax = z.x + m.x, ay = z.y - m.y, bx = z.y + m.y, by = m.x - z.x;
    loc += T(0.25) * (sa * (ax * ax + ay * ay) + sb * (bx * bx + by * by));
    const T hp = T(0.5) * (sa + sb), hm = T(0.5) * (sa - sb);
    v[r].x = hp * z.x + hm * m.x;
    v[r].y = hp * z.y - hm * m.y;
  }
  return loc;
}

// Wavenumber with the Nyquist index zeroed, for a runtime axis length n.
__device__ __forceinline__ int kwave_rt(int i, int n) {
  return (i < n / 2) ? i : (i == n / 2 ? 0 : i - n);
}

// Two derivatives in a row: v (real pencils packed, layout A) is replaced by
// L^2 d(kappa d v) with kappa loaded from kap at layout A positions.
// When kred is given, sum kappa (L d v)^2 over the pencil pair into *kred.
template <typename T, int L, bool CONTIG>
__device__ __forceinline__ void second_derivative_a(cpx<T>* v, cpx<T>* sm, int t, const cpx<T>* twA,
                                                    const cpx<T>* twB, const T* __restrict__ kap,
                                                    long long b0, long long b1, long long st, bool act,
                                                    T* kred = nullptr) {
  constexpr int R = Shape<L>::R;
  fft_ab<T, L, -1>(v, sm, t, twA);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
  fft_ba<T, L, +1>(v, sm, t, twB);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    cpx<T> k = act ? ld2<T, CONTIG>(kap, b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
    if (kred) *kred += k.x * v[r].x * v[r].x + k.y * v[r].y * v[r].y;
    v[r].x *= k.x;
    v[r].y *= k.y;
  }
  fft_ab<T, L, -1>(v, sm, t, twA);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
  fft_ba<T, L, +1>(v, sm, t, twB);
}

// ------------------------------------------------------------ operator pass
// out = a_self * u + acc_in + coef * d_axis(kappa d_axis u)
// coef = c0 * (use_kf ? k_f : 1) * s.  Optional reduction of
// sum kappa (L d_axis u)^2 (the axis's share of (u, (I - sA) u)).
template <typename T>
struct OpArgs {
  const T* u;
  const T* kappa;
  const T* acc_in;   // may be null
  T* out;
  double c0;
  int use_kf;
  int a_self;        // 0 or 1
  int reduce;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  Fin fin;
  const int* tiles;        // strided TMA passes: tiles where kappa is not
  const int* ntiles_act;   // identically zero (null: all tiles)
};

template <typename T, int L, bool CONTIG>
__global__ void __launch_bounds__(kThreads) k_op(OpArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const T coef = T(a.c0 * (a.use_kf ? a.prm->k_f : 1.0) * a.prm->s / (double(L) * double(L)));
  double red = 0.0;
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<CONTIG>(a.g, a.axis, act ? pair : 0, b0, b1, st);
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[r] = act ? ld2<T, CONTIG>(a.u, b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
    T kred = T(0);
    second_derivative_a<T, L, CONTIG>(v, sm, t, a.twA, a.twB, a.kappa, b0, b1, st, act,
                                      a.reduce ? &kred : nullptr);
    red += double(kred);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long off = (long long)idx_a<L>(r, t) * st;
        cpx<T> o = {coef * v[r].x, coef * v[r].y};
        if (a.a_self) o = o + ld2<T, CONTIG>(a.u, b0, b1, off);
        if (a.acc_in) o = o + ld2<T, CONTIG>(a.acc_in, b0, b1, off);
        st2<T, CONTIG>(a.out, b0, b1, off, o);
      }
    }
  }
  if (a.reduce) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

// ---------------------------------------------------------- Hartley passes
enum DhtMode {
  kDhtPlain = 0,   // out = H_axis(in)                              (axis 1)
  kDhtSetup = 1,   // ff = ||in||^2 ; out = H_2(in)                 (axis 2)
  kDhtUpdate = 2,  // r -= alpha q; rr; out = H_2(r)                (axis 2)
  kDhtSym = 3      // out = H_0 S' H_0 in = F_0^-1 S' F_0 in; rz = sum S' (H_0 in)^2   (axis 0)
};

template <typename T>
struct DhtArgs {
  const T* in;
  T* out;
  T* x;          // unused by the passes (kept for callers' convenience)
  const T* p;
  T* r;          // update mode
  const T* q;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;
  Fin fin;
};

template <typename T, int L, bool CONTIG, int MODE>
__global__ void __launch_bounds__(kThreads) k_dht(DhtArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  double red = 0.0;
  T alpha = T(0);
  double symc = 0.0, inv_nn = 0.0;
  if (MODE == kDhtUpdate) alpha = T(a.st->alpha);
  if (MODE == kDhtSym) {
    symc = a.prm->s * a.prm->k_f * a.prm->kbar1;
    inv_nn = a.prm->inv_nn;
  }
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<CONTIG>(a.g, a.axis, act ? pair : 0, b0, b1, st);
    cpx<T> v[R];
    T loc = T(0);
    if (MODE == kDhtUpdate) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cpx<T> rv = {T(0), T(0)};
        if (act) {
          const long long off = (long long)idx_a<L>(r, t) * st;
          const cpx<T> qv = ld2<T, CONTIG>(a.q, b0, b1, off);
          rv = ld2<T, CONTIG>(a.r, b0, b1, off);
          rv.x -= alpha * qv.x;
          rv.y -= alpha * qv.y;
          st2<T, CONTIG>(a.r, b0, b1, off, rv);
          loc += rv.x * rv.x + rv.y * rv.y;
        }
        v[r] = rv;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        v[r] = act ? ld2<T, CONTIG>(a.in, b0, b1, (long long)idx_a<L>(r, t) * st) : cpx<T>{T(0), T(0)};
        if (MODE == kDhtSetup) loc += v[r].x * v[r].x + v[r].y * v[r].y;
      }
    }
    fft_ab<T, L, -1>(v, sm, t, a.twA);
    if (MODE != kDhtSym) hartley_combine<T, L, true>(v, t);
    if (MODE == kDhtSym) {
      // pencils (i1, i2) and (i1, i2 + 1) along axis 0
      const long long P = 2 * (act ? pair : 0);
      const int i1 = int(P / a.g.n[2]), i2 = int(P % a.g.n[2]);
      const int k1 = kwave_rt(i1, a.g.n[1]), k2a = kwave_rt(i2, a.g.n[2]), k2b = kwave_rt(i2 + 1, a.g.n[2]);
      const T base_a = T(k1 * k1 + k2a * k2a);
      const T base_b = T(k1 * k1 + k2b * k2b);
      loc += sym_apply<T, L>(v, t, base_a, base_b, T(symc), T(inv_nn));
      fft_ba<T, L, +1>(v, sm, t, a.twB);
      if (act) {
#pragma unroll
        for (int r = 0; r < R; ++r) st2<T, CONTIG>(a.out, b0, b1, (long long)idx_a<L>(r, t) * st, v[r]);
      }
    } else {
      if (act) {
#pragma unroll
        for (int r = 0; r < R; ++r) st2<T, CONTIG>(a.out, b0, b1, (long long)idx_b<L>(r, t) * st, v[r]);
      }
    }
    if (act) red += double(loc);
  }
  if (MODE != kDhtPlain) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

// --------------------------------------------- PCG direction + operator (x)
// z = H_2(w) (last factor of M^-1 r, scale folded into S'); p = z + beta p;
// q = p - s k_f d_2(kappa d_2 p).  Fields are written at layout-B positions
// of each pencil, which is just a permutation inside the pencil.
// The CG iterate's update x += alpha p is deferred by one iteration: the
// direction kernel of the next iteration applies it while it holds the old p
// (alpha is still the previous iteration's there), and k_cg_final applies the
// last one after the loop; the update kernel then moves only r and q.  The
// sum of alpha_k p_k is formed in the same order as without the deferral.
template <typename T>
struct PcgOpxArgs {
  const T* w;
  T* p;
  T* q;
  T* x;          // CG iterate (deferred update; null: none)
  const T* kappa;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;
  Fin fin;   // reduces |p|^2 and sum kappa (L d_2 p)^2 (kFinPqAdd)
  const int* rowact;   // TMA row tiles: 0 where kappa vanishes on the tile (null: all)
};

template <typename T, int L>
__global__ void __launch_bounds__(kThreads) k_pcg_opx(PcgOpxArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const double betad = a.st->beta;
  const T beta = T(betad);
  // from the second iteration on (st->it counts completed iterations): the
  // previous iteration's x += alpha p with the old p read here anyway
  const bool xupd = a.x && a.st->it > 0;
  const T alpha = xupd ? T(a.st->alpha) : T(0);
  const T coef = T(-a.prm->s * a.prm->k_f / (double(L) * double(L)));
  double red_pp = 0.0, red_k = 0.0;
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<true>(a.g, 2, act ? pair : 0, b0, b1, st);
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = act ? ld2<T, true>(a.w, b0, b1, idx_a<L>(r, t)) : cpx<T>{T(0), T(0)};
    fft_ab<T, L, -1>(v, sm, t, a.twA);
    hartley_combine<T, L, true>(v, t);
    T lpp = T(0), lk = T(0);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long off = idx_b<L>(r, t);
        if (betad != 0.0 || xupd) {
          const cpx<T> po = ld2<T, true>(a.p, b0, b1, off);
          v[r].x += beta * po.x;
          v[r].y += beta * po.y;
          if (xupd) {
            cpx<T> xv = ld2<T, true>(a.x, b0, b1, off);
            xv.x += alpha * po.x;
            xv.y += alpha * po.y;
            st2<T, true>(a.x, b0, b1, off, xv);
          }
        }
        lpp += v[r].x * v[r].x + v[r].y * v[r].y;
        st2<T, true>(a.p, b0, b1, off, v[r]);
      }
    }
    // operator on p, starting from layout B: spectra live in layout A
    fft_ba<T, L, -1>(v, sm, t, a.twB);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_a<L>(r, t)));
    fft_ab<T, L, +1>(v, sm, t, a.twA);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T> k = act ? ld2<T, true>(a.kappa, b0, b1, idx_b<L>(r, t)) : cpx<T>{T(0), T(0)};
      lk += k.x * v[r].x * v[r].x + k.y * v[r].y * v[r].y;
      v[r].x *= k.x;
      v[r].y *= k.y;
    }
    red_pp += double(lpp);
    red_k += double(lk);
    fft_ba<T, L, -1>(v, sm, t, a.twB);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_a<L>(r, t)));
    fft_ab<T, L, +1>(v, sm, t, a.twA);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long off = idx_b<L>(r, t);
        cpx<T> pv = ld2<T, true>(a.p, b0, b1, off);
        st2<T, true>(a.q, b0, b1, off, {pv.x + coef * v[r].x, pv.y + coef * v[r].y});
      }
    }
  }
  double vv[2] = {red_pp, red_k};
  reduce_finish<2>(vv, a.fin);
}

// ----------------------------------------------------------- gradient pass
// sum_x kappa1 d_axis(u0 + u1) d_axis(w) accumulated into the reduction.
template <typename T>
struct GradArgs {
  const T* u0;
  const T* u1;   // may be null
  const T* w;
  const T* kappa;
  T* q;          // optional per-voxel field: q += qscale d_axis(u0 + u1) d_axis(w)
  double qscale;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Fin fin;
  const int* tiles;        // as in OpArgs
  const int* ntiles_act;
};

template <typename T, int L, bool CONTIG>
__global__ void __launch_bounds__(kThreads) k_grad(GradArgs<T> a) {
  using Sh = Shape<L>;
  constexpr int R = Sh::R, TH = Sh::TH, G = Sh::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw) + g * Sh::GSTRIDE;
  const long long npairs = a.g.nn / L / 2;
  const T scale = T(1.0 / (double(L) * double(L)));
  double red = 0.0;
  for (long long base = (long long)blockIdx.x * G; base < npairs; base += (long long)gridDim.x * G) {
    const long long pair = base + g;
    const bool act = pair < npairs;
    long long b0, b1, st;
    pair_addr<CONTIG>(a.g, a.axis, act ? pair : 0, b0, b1, st);
    cpx<T> du[R], dw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const long long off = (long long)idx_a<L>(r, t) * st;
      du[r] = act ? ld2<T, CONTIG>(a.u0, b0, b1, off) : cpx<T>{T(0), T(0)};
      if (a.u1 && act) du[r] = du[r] + ld2<T, CONTIG>(a.u1, b0, b1, off);
      dw[r] = act ? ld2<T, CONTIG>(a.w, b0, b1, off) : cpx<T>{T(0), T(0)};
    }
    fft_ab<T, L, -1>(du, sm, t, a.twA);
#pragma unroll
    for (int r = 0; r < R; ++r) du[r] = times_ik(du[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1>(du, sm, t, a.twB);
    fft_ab<T, L, -1>(dw, sm, t, a.twA);
#pragma unroll
    for (int r = 0; r < R; ++r) dw[r] = times_ik(dw[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1>(dw, sm, t, a.twB);
    if (act) {
      T loc = T(0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cpx<T> k = ld2<T, CONTIG>(a.kappa, b0, b1, (long long)idx_a<L>(r, t) * st);
        loc += k.x * du[r].x * dw[r].x + k.y * du[r].y * dw[r].y;
      }
      red += double(loc * scale);
      if (a.q) {
        const T qs = T(a.qscale) * scale;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const long long off = (long long)idx_a<L>(r, t) * st;
          cpx<T> qv = ld2<T, CONTIG>(a.q, b0, b1, off);
          qv.x += qs * du[r].x * dw[r].x;
          qv.y += qs * du[r].y * dw[r].y;
          st2<T, CONTIG>(a.q, b0, b1, off, qv);
        }
      }
    }
  }
  double vv[1] = {red};
  reduce_finish<1>(vv, a.fin);
}

// -------------------------------------------------------- pointwise kernels
// Strang-split step pieces, element by element.  s = tau/2, e = exp(rho s),
// rho = rho_f * rho1.  "prev" is the state c_n itself (prev_is_state) or the
// c** of the previous step, from which c_n = L_s(c**).
enum PwKind {
  kPwFwdPre = 0,   // out0 = c* = L_s(c_n)
  kPwFwdPost,      // out0 = c** = a + b
  kPwMisfit,       // c1 = L_s(a); acc sum (c1 - d)^2; out0 = d - c1 (alpha(1)); out1 = c1 (opt)
  kPwAdjPre,       // a = alpha_{n+1}, b = c**_n: gacc += alpha rho1 c_{n+1}(1 - c_{n+1});
                   // out0 = alpha** = L_s'(c**) alpha; out1 = c* + c**; out2 = c_n
  kPwAdjPost,      // a = alpha**, b = x, d = r, prev = c_n:  alpha* = a + 2 b + d;
                   // gacc += alpha* rho1 c* (1 - c*); out0 = L_s'(c_n) alpha*
  kPwTlPre,        // a = chat_n, b = c**_n: out0 = chat*, out1 = 2 k_f chat* + v_k (c* + c**)
  kPwTlPost,       // a = chat*, b = x, d = c**_n: out0 = chat_{n+1}
  kPwNeg,          // out0 = -a
  kPwState         // out0 = c_n (the state itself, or L_s of the previous c**)
};

template <typename T>
struct PwArgs {
  const T* a;
  const T* b;
  const T* d;
  const T* prev;
  const T* rho1;
  const T* m[3];    // tissue maps (Moving-Atlas misfit), null when unused
  const T* md[3];   // anatomy data m_D
  T* q;             // adjoint passes: per-voxel rho_f integrand, null when unused
  T* out0;
  T* out1;
  T* out2;
  int prev_is_state;
  long long nn;
  Params* prm;
  int reduce;
  Fin fin;
};

// The input values of one element of a pointwise step (only the ones the
// step reads are loaded).
template <typename T>
struct PwVals {
  T a, b, d, pv, rh, q;
};

template <typename T, int KIND>
__device__ __forceinline__ PwVals<T> pw_load(long long i, const PwArgs<T>& a) {
  constexpr bool A = KIND != kPwFwdPre && KIND != kPwState;
  constexpr bool B = KIND == kPwFwdPost || KIND == kPwAdjPre || KIND == kPwAdjPost || KIND == kPwTlPre ||
                     KIND == kPwTlPost;
  constexpr bool D = KIND == kPwMisfit || KIND == kPwAdjPost || KIND == kPwTlPost;
  constexpr bool PV = KIND == kPwFwdPre || KIND == kPwAdjPre || KIND == kPwAdjPost || KIND == kPwTlPre ||
                      KIND == kPwState;
  constexpr bool Q = KIND == kPwAdjPre || KIND == kPwAdjPost;
  PwVals<T> v{T(0), T(0), T(0), T(0), T(0), T(0)};
  if (KIND != kPwFwdPost && KIND != kPwNeg && !(KIND == kPwState && a.prev_is_state)) v.rh = a.rho1[i];
  if (A) v.a = a.a[i];
  if (B) v.b = a.b[i];
  if (D) v.d = a.d[i];
  if (PV) v.pv = a.prev[i];
  if (Q && a.q) v.q = a.q[i];
  return v;
}

// One element of a pointwise step from its loaded inputs: writes the
// outputs, returns the element's term of the reduction.
template <typename T, int KIND>
__device__ __forceinline__ T pw_compute(long long i, const PwArgs<T>& a, const PwVals<T>& v, T s, T rho_f, T k_f,
                                        T v_k, T v_rho) {
  T term = T(0);
  const T rho1 = v.rh;
  T e = T(1);
  if (KIND != kPwFwdPost && KIND != kPwNeg && !(KIND == kPwState && a.prev_is_state)) e = expT(rho_f * rho1 * s);
  T cn = T(0);
  if (KIND == kPwFwdPre || KIND == kPwAdjPre || KIND == kPwTlPre || KIND == kPwState) {
    cn = v.pv;
    if (!a.prev_is_state) cn = logistic(cn, e);
  }
  if (KIND == kPwFwdPre) {
    a.out0[i] = logistic(cn, e);
  } else if (KIND == kPwFwdPost) {
    a.out0[i] = v.a + v.b;
  } else if (KIND == kPwMisfit) {
    const T c1 = logistic(v.a, e);
    const T dd = v.d;
    const T r = c1 - dd;
    T rr = r * r, al = dd - c1;
    if (a.md[0]) {
      // D_m = 1/2 sum_i (m_i (1 - c) - m_D,i)^2 and its -dD_m/dc
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T mi = a.m[j][i];
        const T ej = mi * (T(1) - c1) - a.md[j][i];
        rr += ej * ej;
        al += mi * ej;
      }
    }
    term += rr;
    a.out0[i] = al;
    if (a.out1) a.out1[i] = c1;
  } else if (KIND == kPwAdjPre) {
    const T al = v.a, css = v.b;
    const T cnext = logistic(css, e);
    term += al * rho1 * cnext * (T(1) - cnext);
    if (a.q) a.q[i] = v.q - s * al * cnext * (T(1) - cnext);
    a.out0[i] = logistic_dc(css, e) * al;
    a.out1[i] = logistic(cn, e) + css;
    a.out2[i] = cn;
  } else if (KIND == kPwAdjPost) {
    const T c = v.pv;
    const T ast = v.a + T(2) * v.b + v.d;
    const T cs = logistic(c, e);
    term += ast * rho1 * cs * (T(1) - cs);
    if (a.q) a.q[i] = v.q - s * ast * cs * (T(1) - cs);
    a.out0[i] = logistic_dc(c, e) * ast;
  } else if (KIND == kPwTlPre) {
    const T css = v.b;
    const T cs = logistic(cn, e);
    const T chs = logistic_dc(cn, e) * v.a + v_rho * s * rho1 * cs * (T(1) - cs);
    a.out0[i] = chs;
    a.out1[i] = T(2) * k_f * chs + v_k * (cs + css);
  } else if (KIND == kPwTlPost) {
    const T css = v.d;
    const T chss = v.a + v.b;
    const T cnext = logistic(css, e);
    a.out0[i] = logistic_dc(css, e) * chss + v_rho * s * rho1 * cnext * (T(1) - cnext);
  } else if (KIND == kPwNeg) {
    T w = T(1);
    if (a.md[0]) {
#pragma unroll
      for (int j = 0; j < 3; ++j) w += a.m[j][i] * a.m[j][i];
    }
    a.out0[i] = -w * v.a;
  } else if (KIND == kPwState) {
    a.out0[i] = cn;
  }
  return term;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) k_pw(PwArgs<T> a) {
  const double sd = a.prm->s;
  const T s = T(sd), rho_f = T(a.prm->rho_f);
  const T k_f = T(a.prm->k_f), v_k = T(a.prm->v_k), v_rho = T(a.prm->v_rho);
  double red = 0.0;
  // four elements per thread and trip, a grid stride apart (every load stays
  // coalesced): the inputs of all four are loaded before any is computed, so
  // their loads are in flight together; the reduced terms of the four are
  // summed in T, then added in FP64
  const long long gs = (long long)gridDim.x * kThreads;
  for (long long i0 = (long long)blockIdx.x * kThreads + threadIdx.x; i0 < a.nn; i0 += 4 * gs) {
    T loc = T(0);
    if (i0 + 3 * gs < a.nn) {
      PwVals<T> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = pw_load<T, KIND>(i0 + u * gs, a);
#pragma unroll
      for (int u = 0; u < 4; ++u) loc += pw_compute<T, KIND>(i0 + u * gs, a, v[u], s, rho_f, k_f, v_k, v_rho);
    } else {
      for (long long i = i0; i < a.nn; i += gs)
        loc += pw_compute<T, KIND>(i, a, pw_load<T, KIND>(i, a), s, rho_f, k_f, v_k, v_rho);
    }
    red += double(loc);
  }
  if (a.reduce) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

// ------------------------------------------------ coefficients, conversion
// kappa1 = sum_i k_i m_i, rho1 = sum_i rho_i m_i (Eq. coeff_tumor) from FP64
// tissue maps; sum(kappa1) reduced for the preconditioner constant.
template <typename T>
struct CoefArgs {
  const double* m0;
  const double* m1;
  const double* m2;
  T* kappa1;
  T* rho1;
  double kw0, kw1, kw2, rw0, rw1, rw2;
  long long nn;
  Fin fin;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_coef(CoefArgs<T> a) {
  double red = 0.0, cnt = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.nn;
       i += (long long)gridDim.x * kThreads) {
    const double x0 = a.m0[i], x1 = a.m1[i], x2 = a.m2[i];
    const double k = a.kw0 * x0 + a.kw1 * x1 + a.kw2 * x2;
    a.kappa1[i] = T(k);
    a.rho1[i] = T(a.rw0 * x0 + a.rw1 * x1 + a.rw2 * x2);
    if (k > 0.0) {
      red += double(T(k));
      cnt += 1.0;
    }
  }
  double vv[2] = {red, cnt};
  reduce_finish<2>(vv, a.fin);
}

// ||x + cy y||^2 (y may be null) reduced in FP64 into the Fin target: the
// squared norm of a Crank-Nicolson right-hand side for the PCG stopping test.
template <typename T>
struct NormArgs {
  const T* x;
  const T* y;
  double cy;
  long long nn;
  Fin fin;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_normsq(NormArgs<T> a) {
  double red = 0.0;
  const T c = T(a.cy);
  // as in k_pw: four elements per trip, squares summed in T, then in FP64
  const long long gs = (long long)gridDim.x * kThreads;
  for (long long i0 = (long long)blockIdx.x * kThreads + threadIdx.x; i0 < a.nn; i0 += 4 * gs) {
    auto sq = [&](long long i) {
      T v = a.x[i];
      if (a.y) v += c * a.y[i];
      return v * v;
    };
    T loc = T(0);
    if (i0 + 3 * gs < a.nn) {
#pragma unroll
      for (int u = 0; u < 4; ++u) loc += sq(i0 + u * gs);
    } else {
      for (long long i = i0; i < a.nn; i += gs) loc += sq(i);
    }
    red += double(loc);
  }
  double vv[1] = {red};
  reduce_finish<1>(vv, a.fin);
}

// Start of a solve: x = 0, unless the solve starts from a guess already in
// x (st->keep_x, set on the stream before the solve).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_x_init(T* __restrict__ x, const PcgState* st, long long nn) {
  if (st->keep_x) return;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads)
    x[i] = T(0);
}

// Initial guess of a state solve (I - sA) x = f from the increments of the
// previous one or two time steps, extrapolated in time, with its residual
// taken from their stored images g = (I - sA) d, so that no operator is
// applied:  order 0: x = 0, r = f;  order 1: x = d1, r = f - g1;
// order 2: x = 2 d1 - d2, r = f - (2 g1 - g2).  f comes in r and is kept in fs.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_guess(T* __restrict__ r, T* __restrict__ x, T* __restrict__ fs,
                                                    const T* __restrict__ d1, const T* __restrict__ d2,
                                                    const T* __restrict__ g1, const T* __restrict__ g2, int order,
                                                    long long nn) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads) {
    const T f = r[i];
    fs[i] = f;
    if (order >= 2) {
      x[i] = T(2) * d1[i] - d2[i];
      r[i] = f - (T(2) * g1[i] - g2[i]);
    } else if (order == 1) {
      x[i] = d1[i];
      r[i] = f - g1[i];
    } else {
      x[i] = T(0);
    }
  }
}

// After a state solve: d = x and g = f - r, which is (I - sA) x up to the
// rounding of the residual recursion.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_guess_keep(T* __restrict__ d, T* __restrict__ g,
                                                         const T* __restrict__ x, const T* __restrict__ r,
                                                         const T* __restrict__ fs, long long nn) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads) {
    d[i] = x[i];
    g[i] = fs[i] - r[i];
  }
}

// The last deferred CG update after the iteration loop: x += alpha p when
// at least one iteration ran.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_final(T* __restrict__ x, const T* __restrict__ p,
                                                       const PcgState* st, long long nn) {
  if (st->it <= 0) return;
  const T alpha = T(st->alpha);
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads)
    x[i] += alpha * p[i];
}

// out = ca qk + cb qr in FP64 (coupling field of one tissue class)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_combine(const T* __restrict__ qk, const T* __restrict__ qr,
                                                      double ca, double cb, double* __restrict__ out,
                                                      long long nn) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads)
    out[i] = ca * double(qk[i]) + cb * double(qr[i]);
}

template <typename TO, typename TI>
__global__ void __launch_bounds__(kThreads) k_convert(const TI* __restrict__ in, TO* __restrict__ out,
                                                      long long nn, double scale) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < nn; i += (long long)gridDim.x * kThreads)
    out[i] = TO(double(in[i]) * scale);
}

// ---------------------------------------------------------- Gaussian basis
// G_i(x) = g_i0(x0) g_i1(x1) g_i2(x2) with per-axis factor tables
// fac[(i * 3 + a) * nmax + x] = exp(-d_a(x)^2 / (2 sigma^2)), d_a the
// minimum-image distance (Eq. tumor:fwd-init; Sec. 4.1).
template <typename T>
struct PhiArgs {
  const double* fac;   // np * 3 * nmax
  const T* fac_t;      // the same factors in T
  const double* p;     // np (device)
  T* out;              // synthesis output
  const T* u;          // projection input
  double* part;        // projection partials: np * n0
  int np, nmax;
  Geom g;
  double cut;          // factors below cut are skipped
};

// c(0) = sum_i p_i G_i: one block per (x0, x1) row; the row coefficients
// p_i g_i0(x0) g_i1(x1) are staged in shared memory and summed in basis
// order, so the result is deterministic.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_phi(PhiArgs<T> a) {
  extern __shared__ double coef_raw[];   // np doubles; holds np values of T
  T* coef = reinterpret_cast<T*>(coef_raw);
  const int n0 = a.g.n[0], n1 = a.g.n[1], n2 = a.g.n[2];
  for (long long row = blockIdx.x; row < (long long)n0 * n1; row += gridDim.x) {
    const int x0 = int(row / n1), x1 = int(row % n1);
    int any = 0;
    for (int i = threadIdx.x; i < a.np; i += kThreads) {
      double c = a.p[i] * a.fac[(i * 3 + 0) * a.nmax + x0] * a.fac[(i * 3 + 1) * a.nmax + x1];
      if (!(fabs(c) > a.cut)) c = 0.0;
      coef[i] = T(c);
      any |= (c != 0.0);
    }
    any = __syncthreads_or(any);
    // the field is stored in T, so the sum over the basis runs in T too
    for (int x2 = threadIdx.x; x2 < n2; x2 += kThreads) {
      T s = T(0);
      if (any) {
        for (int i = 0; i < a.np; ++i) {
          const T c = coef[i];
          if (c != T(0)) s += c * a.fac_t[(i * 3 + 2) * a.nmax + x2];
        }
      }
      a.out[row * n2 + x2] = s;
    }
    __syncthreads();
  }
}

// (Phi^T u)_i partials: block (i, x0) sums g_i0(x0) g_i1(x1) g_i2(x2) u over
// (x1, x2); a second kernel adds the n0 partials of each i in order.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_phit(PhiArgs<T> a) {
  const int i = blockIdx.y;
  const int n0 = a.g.n[0], n1 = a.g.n[1], n2 = a.g.n[2];
  for (int x0 = blockIdx.x; x0 < n0; x0 += gridDim.x) {
    const double f0 = a.fac[(i * 3 + 0) * a.nmax + x0];
    double s = 0.0;
    if (fabs(f0) > a.cut) {
      for (int x1 = threadIdx.x / 32; x1 < n1; x1 += kWarps) {
        const double f1 = a.fac[(i * 3 + 1) * a.nmax + x1];
        if (fabs(f0 * f1) <= a.cut) continue;
        // one lane's share of a row (n2 / 32 terms) is summed in T
        T r = T(0);
        const T* row = a.u + ((long long)x0 * n1 + x1) * n2;
        for (int x2 = threadIdx.x & 31; x2 < n2; x2 += 32) r += a.fac_t[(i * 3 + 2) * a.nmax + x2] * row[x2];
        s += f0 * f1 * double(r);
      }
    }
    double vv = warp_sum(s);
    __shared__ double sw[kWarps];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = vv;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < kWarps; ++w) tot += sw[w];
      a.part[(long long)i * n0 + x0] = tot;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_phit_sum(const double* part, double* out, int np, int n0, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double s = 0.0;
  for (int x0 = 0; x0 < n0; ++x0) s += part[(long long)i * n0 + x0];
  out[i] = scale * s;
}

}  // namespace rd
