// Device-side building blocks shared by every kernel of the library:
// complex arithmetic, grid geometry, the device-resident solver state and
// the deterministic FP64 block reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rd {

constexpr int kThreads = 256;   // threads per block of every field kernel
constexpr int kWarps = kThreads / 32;

// Complex value; aligned to its full size so that tables and buffers of
// cpx<double> can be read with 16-byte vector loads.
template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }

// a * w with w = (c, s)
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, T c, T s) {
  return {a.x * c - a.y * s, a.x * s + a.y * c};
}

// Grid: n[0] x n[1] x n[2], n[2] fastest (C order), periodic box [0, 2 pi)^3.
struct Geom {
  int n[3];
  long long nn;
};

// Scalars of one preconditioned CG solve, resident on the device so that the
// iteration can run without host round trips.
struct PcgState {
  double ff;      // ||f||^2, f = right-hand side of the increment system
  double bb;      // ||b||^2, b = right-hand side of the Crank-Nicolson system
                  // (0: the stopping test uses ff)
  double rr;      // ||r||^2
  double rz;      // (r, M^-1 r)
  double pq;      // (p, (I - sA) p)
  double pq_part; // partial sums of pq from the passes before the last
  double alpha, beta;
  double rtol2;   // rtol^2
  int it, maxit, done, status;
  int total_it;   // iterations summed over all solves since reset
  int sticky;     // largest status seen since reset
  int keep_x;     // 1: the solve starts from the guess already in x (set before its setup)
};

// Per-call scalars (device resident so that captured launches stay valid).
struct Params {
  double k_f, rho_f;
  double s;        // tau / 2
  double kbar1;    // mean of kappa1 = sum_i k_i m_i
  double v_k, v_rho;
  double h3;
  double inv_nn;   // 1 / (n0 n1 n2)
  double acc[8];   // FP64 accumulators: see kAcc*
};

enum AccSlot {
  kAccMisfit = 0,   // sum (c(1) - d)^2
  kAccGk = 1,       // sum kappa1 grad(abar) . grad(c* + c**)
  kAccGrho = 2,     // sum rho1 alpha L (1 - L)
  kAccGp = 3        // unused placeholder
};

enum StatusCode {
  kStOk = 0,
  kStNoConv = 5,
  kStNonFinite = 6,
  kStTimeout = 7     // a bounded device-side wait gave up
};

enum FinKind {
  kFinNone = 0,
  kFinAcc,      // prm->acc[slot] += scale * total
  kFinSetup,    // start of a solve: ff = rr = total
  kFinRz,       // rz update and beta
  kFinPq,       // alpha
  kFinRr,       // residual norm, iteration count, convergence
  kFinSet,      // *target = scale * total
  kFinPqAdd,    // pq_part += [tot0] + scale s k_f tot_last   (p.p and kappa |d p|^2 terms)
  kFinPqLast,   // pq = pq_part + scale s k_f tot; alpha = rz / pq
  kFinRatio     // *target = total_0 / total_1 (0 when total_1 == 0)
};

struct Fin {
  int kind;
  int slot;
  double scale;
  PcgState* st;
  Params* prm;
  double* part;            // per-block partials
  unsigned int* counter;   // completion counter (reset by the last block)
  double* target;          // kFinSet destination
  unsigned long long cond; // graph WHILE-node handle set to "not done" (0: none)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (p, (I - s A) p) = |p|^2 + s k_f sum_a sum_x kappa1 (d_a p)^2 (the
// spectral first derivative is antisymmetric), accumulated pass by pass.
__device__ __forceinline__ double pq_term(const Fin& f, const double* tot, int K) {
  return (K >= 2 ? tot[0] : 0.0) + tot[K - 1] * f.scale * f.prm->s * f.prm->k_f;
}

__device__ __forceinline__ void finalize(const Fin& f, const double* tots, int K) {
  PcgState* st = f.st;
  const double tot = tots[0];
  switch (f.kind) {
    case kFinAcc:
      for (int k = 0; k < K; ++k) f.prm->acc[f.slot + k] += f.scale * tots[k];
      break;
    case kFinSetup:
      st->ff = tot;
      st->rr = tot;
      st->it = 0;
      st->rz = 0.0;
      st->beta = 0.0;
      st->alpha = 0.0;
      st->pq = 1.0;
      st->pq_part = 0.0;
      st->status = isfinite(tot) ? kStOk : kStNonFinite;
      st->done = (tot > 0.0 && isfinite(tot)) ? 0 : 1;
      if (st->status > st->sticky) st->sticky = st->status;
      if (f.cond) cudaGraphSetConditional(f.cond, st->done ? 0u : 1u);
      break;
    case kFinRz: {
      double rz_new = tot;
      st->beta = (st->it == 0 || st->rz == 0.0) ? 0.0 : rz_new / st->rz;
      st->rz = rz_new;
      if (!isfinite(rz_new)) { st->done = 1; st->status = kStNonFinite; st->sticky = kStNonFinite; }
      break;
    }
    case kFinPq:
      st->pq = tot;
      st->alpha = (tot > 0.0) ? st->rz / tot : 0.0;
      if (!isfinite(tot)) { st->done = 1; st->status = kStNonFinite; }
      break;
    case kFinPqAdd:
      st->pq_part += pq_term(f, tots, K);
      break;
    case kFinPqLast: {
      const double pq = st->pq_part + pq_term(f, tots, K);
      st->pq_part = 0.0;
      st->pq = pq;
      st->alpha = (pq > 0.0) ? st->rz / pq : 0.0;
      if (!isfinite(pq)) { st->done = 1; st->status = kStNonFinite; }
      break;
    }
    case kFinRr:
      st->rr = tot;
      st->it += 1;
      st->total_it += 1;
      if (st->sticky == kStTimeout) {
        st->done = 1;
      } else if (!isfinite(tot) || st->status == kStNonFinite) {
        st->done = 1;
        st->status = kStNonFinite;
      } else if (tot <= st->rtol2 * (st->bb > 0.0 ? st->bb : st->ff)) {
        st->done = 1;
      } else if (st->it >= st->maxit || !(st->pq > 0.0)) {
        st->done = 1;
        st->status = kStNoConv;
      }
      if (st->status > st->sticky) st->sticky = st->status;
      if (f.cond) cudaGraphSetConditional(f.cond, st->done ? 0u : 1u);
      break;
    case kFinSet:
      *f.target = f.scale * tot;
      break;
    case kFinRatio:
      *f.target = (K > 1 && tots[1] > 0.0) ? tots[0] / tots[1] : 0.0;
      break;
    default:
      break;
  }
}

// Deterministic block + grid reduction of K values.  Every thread of the
// block must call it.  The last block to finish sums the per-block partials
// in a fixed order and applies the finaliser, so the result does not depend
// on block scheduling.
template <int K>
__device__ __forceinline__ void reduce_finish(double (&v)[K], const Fin& f) {
  __shared__ double s[K][32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = warp_sum(v[k]);
    if (lane == 0) s[k][w] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int i = 0; i < nw; ++i) t += s[k][i];
      f.part[blockIdx.x * K + k] = t;
    }
    __threadfence();
    unsigned int prev = atomicAdd(f.counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(&f.part[b * K + k]);
    t = warp_sum(t);
    tot[k] = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (lane == 0) s[k][w] = tot[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int i = 0; i < nw; ++i) t += s[k][i];
      tot[k] = t;
    }
    finalize(f, tot, K);
    *f.counter = 0u;
  }
}

// Exact logistic flow of dc/dt = rho c (1 - c) over time t, and its
// derivative with respect to the initial value (Sec. 3.3, analytic reaction).
template <typename T>
__device__ __forceinline__ T logistic(T c, T e) {   // e = exp(rho t)
  return c * e / (T(1) - c + c * e);
}
template <typename T>
__device__ __forceinline__ T logistic_dc(T c, T e) {
  T d = T(1) - c + c * e;
  return e / (d * d);
}
__device__ __forceinline__ float expT(float x) { return expf(x); }
__device__ __forceinline__ double expT(double x) { return exp(x); }

}  // namespace rd
