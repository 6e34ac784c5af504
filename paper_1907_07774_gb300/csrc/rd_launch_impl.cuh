// Definitions of the launchers; included once per precision.
#pragma once

#include <mutex>
#include <unordered_map>

#include "rd_launch.cuh"

namespace rd {

namespace detail {

inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Blocks that fit on the device at once for a kernel (persistent grid size),
// cached per kernel; also raises the dynamic shared-memory limit when needed.
inline int resident_blocks(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) return it->second;
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem) != cudaSuccess || occ < 1) occ = 1;
  int nb = occ * sm_count();
  if (nb > kMaxBlocks) nb = kMaxBlocks;
  cache[fn] = nb;
  return nb;
}

inline int grid_for(const void* fn, size_t smem, long long work_items) {
  int cap = resident_blocks(fn, smem);
  long long want = work_items < 1 ? 1 : work_items;
  return (int)(want < cap ? want : cap);
}

template <typename T, int L>
constexpr size_t pencil_smem() {
  return size_t(Shape<L>::G) * Shape<L>::GSTRIDE * sizeof(cpx<T>);
}

template <typename K, typename A>
cudaError_t launch_pencil(K kern, size_t smem, long long groups_needed, const A& a, cudaStream_t s,
                          int cls = kcOther, int L = 0) {
  const void* fn = reinterpret_cast<const void*>(kern);
  int grid = grid_for(fn, smem, groups_needed);
  const int tc = tuned_cap(cls, L);
  if (tc > 0 && tc < grid) grid = tc;
  const int tok = prof_begin(cls, s);
  kern<<<grid, kThreads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  prof_end(tok, s);
  return e;
}

#define RD_DISPATCH_L(L, ...)                          \
  switch (L) {                                         \
    case 8: { constexpr int LL = 8; __VA_ARGS__ }      \
    case 16: { constexpr int LL = 16; __VA_ARGS__ }    \
    case 32: { constexpr int LL = 32; __VA_ARGS__ }    \
    case 64: { constexpr int LL = 64; __VA_ARGS__ }    \
    case 96: { constexpr int LL = 96; __VA_ARGS__ }    \
    case 128: { constexpr int LL = 128; __VA_ARGS__ }  \
    case 256: { constexpr int LL = 256; __VA_ARGS__ }  \
    default: return cudaErrorInvalidValue;             \
  }

}  // namespace detail

namespace detail {
template <typename T>
inline bool tma_fits(const Geom& g) {
  const int W = 64 / int(sizeof(T));
  return g.n[2] % W == 0;
}
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename K, typename A>
cudaError_t launch_tma(K kern, size_t smem, int threads, long long tiles, const A& a, cudaStream_t s, int cls,
                       int L) {
  const void* fn = reinterpret_cast<const void*>(kern);
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int cap;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it == cache.end()) {
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) occ = 1;
      cap = occ * sm_count();
      if (cap > kMaxBlocks) cap = kMaxBlocks;
      cache[fn] = cap;
    } else {
      cap = it->second;
    }
  }
  const int tc = tuned_cap(cls, L);
  if (tc > 0 && tc < cap) cap = tc;
  const int grid = (int)(tiles < cap ? tiles : cap);
  const int tok = prof_begin(cls, s);
  kern<<<grid, threads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  prof_end(tok, s);
  return e;
}
}  // namespace detail

template <typename T>
cudaError_t Launch<T>::op(int L, const OpArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  const long long npairs = a.g.nn / L / 2;
  if (a.axis == 2 && !tuned_pencil(kcOpContig, L) && a.a_self == 0 && !a.acc_in && !a.reduce && a.out && a.fin.st &&
      aligned16(a.u) &&
      aligned16(a.kappa) && aligned16(a.out)) {
    RD_DISPATCH_L(L, {
      using TS = TmaRowShape<T, LL>;
      if constexpr (TS::OK) {
        const long long rows = a.g.nn / LL;
        OpRowTmaArgs<T> t;
        if (rows % TS::ROWS == 0 && row_map(&t.map_u, a.u, a.g, sizeof(T), TS::ROWS) &&
            row_map(&t.map_k, a.kappa, a.g, sizeof(T), TS::ROWS)) {
          t.out = a.out;
          t.c0 = a.c0;
          t.use_kf = a.use_kf;
          t.g = a.g;
          t.twA = a.twA;
          t.twB = a.twB;
          t.prm = a.prm;
          t.st = a.fin.st;
          return launch_tma(k_op_row_tma<T, LL>, TS::OPROW_SMEM, TS::THREADS, rows / TS::ROWS, t, s, kcOpContig, LL);
        }
      }
      break;
    })
  }
  if (a.axis != 2 && !tuned_pencil(kcOpStrided, L) && a.a_self == 0 && a.acc_in == a.out && a.out &&
      tma_fits<T>(a.g) && aligned16(a.u) &&
      aligned16(a.kappa) && aligned16(a.out)) {
    RD_DISPATCH_L(L, {
      using TS = TmaShape<T, LL>;
      if constexpr (TS::OK) {
        OpTmaArgs<T> t;
        if (strided_map(&t.map_u, a.u, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_k, a.kappa, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_q, a.out, a.g, sizeof(T), a.axis)) {
          t.c0 = a.c0;
          t.use_kf = a.use_kf;
          t.reduce = a.reduce;
          t.axis = a.axis;
          t.g = a.g;
          t.twA = a.twA;
          t.twB = a.twB;
          t.prm = a.prm;
          t.st = a.fin.st;
          t.fin = a.fin;
          t.tiles = a.tiles;
          t.ntiles_act = a.ntiles_act;
          const long long tiles = (long long)(a.g.n[2] / TS::W) * (a.axis == 1 ? a.g.n[0] : a.g.n[1]);
          if constexpr (sizeof(T) == 4) {
            if (a.axis == 1)
              return launch_tma(k_op_tma_red<T, LL, 1>, TS::OPR_SMEM, TS::THREADS, tiles, t, s, kcOpStrided, LL);
            return launch_tma(k_op_tma_red<T, LL, 0>, TS::OPR_SMEM, TS::THREADS, tiles, t, s, kcOpStrided, LL);
          } else {
            if (a.axis == 1) return launch_tma(k_op_tma<T, LL, 1>, TS::OP_SMEM, TS::THREADS, tiles, t, s, kcOpStrided, LL);
            return launch_tma(k_op_tma<T, LL, 0>, TS::OP_SMEM, TS::THREADS, tiles, t, s, kcOpStrided, LL);
          }
        }
      }
      break;
    })
  }
  RD_DISPATCH_L(L, {
    constexpr size_t sm = pencil_smem<T, LL>();
    const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
    if (a.axis == 2) return launch_pencil(k_op<T, LL, true>, sm, blocks, a, s, kcOpContig, LL);
    return launch_pencil(k_op<T, LL, false>, sm, blocks, a, s, kcOpStrided, LL);
  })
}

template <typename T>
cudaError_t Launch<T>::dht(int L, int mode, const DhtArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  const long long npairs = a.g.nn / L / 2;
  if (a.axis == 2 && (mode == kDhtSetup || mode == kDhtUpdate) &&
      !tuned_pencil(mode == kDhtSetup ? kcDhtSetup : kcDhtUpdate, L)) {
    const void* rr = (mode == kDhtSetup) ? (const void*)a.in : (const void*)a.r;
    const bool al = aligned16(rr) && aligned16(a.out) && (mode == kDhtSetup || aligned16(a.q));
    if (al) {
      RD_DISPATCH_L(L, {
        using TS = TmaRowShape<T, LL>;
        if constexpr (TS::OK) {
          const long long rows = a.g.nn / LL;
          DhtRowTmaArgs<T> t;
          bool ok = rows % TS::ROWS == 0 && row_map(&t.map_r, rr, a.g, sizeof(T), TS::ROWS) &&
                    row_map(&t.map_out, a.out, a.g, sizeof(T), TS::ROWS);
          if (ok && mode == kDhtUpdate)
            ok = row_map(&t.map_q, a.q, a.g, sizeof(T), TS::ROWS);
          else if (ok)
            t.map_q = t.map_r;
          if (ok) {
            t.g = a.g;
            t.twA = a.twA;
            t.twB = a.twB;
            t.st = a.st;
            t.fin = a.fin;
            const long long tiles = rows / TS::ROWS;
            if (mode == kDhtUpdate)
              return launch_tma(k_dht_row_tma<T, LL, kDhtUpdate>, TS::UPD_SMEM, TS::THREADS, tiles, t, s, kcDhtUpdate, LL);
            return launch_tma(k_dht_row_tma<T, LL, kDhtSetup>, TS::SETUP_SMEM, TS::THREADS, tiles, t, s, kcDhtSetup, LL);
          }
        }
        break;
      })
    }
  }
  if (a.axis != 2 && (mode == kDhtPlain || mode == kDhtSym) && !tuned_pencil(mode == kDhtSym ? kcDhtSym : kcDhtPlain, L) &&
      tma_fits<T>(a.g) && aligned16(a.in) &&
      aligned16(a.out)) {
    RD_DISPATCH_L(L, {
      using TS = TmaShape<T, LL>;
      if constexpr (TS::OK) {
        DhtTmaArgs<T> t;
        if (strided_map(&t.map_in, a.in, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_out, a.out, a.g, sizeof(T), a.axis)) {
          t.axis = a.axis;
          t.g = a.g;
          t.twA = a.twA;
          t.twB = a.twB;
          t.prm = a.prm;
          t.st = a.st;
          t.fin = a.fin;
          const long long tiles = (long long)(a.g.n[2] / TS::W) * (a.axis == 1 ? a.g.n[0] : a.g.n[1]);
          const int cls = (mode == kDhtSym) ? kcDhtSym : kcDhtPlain;
          if (mode == kDhtSym) {
            if (a.axis == 1) return launch_tma(k_dht_tma<T, LL, 1, kDhtSym>, TS::DHT_SMEM, TS::THREADS, tiles, t, s, cls, LL);
            return launch_tma(k_dht_tma<T, LL, 0, kDhtSym>, TS::DHT_SMEM, TS::THREADS, tiles, t, s, cls, LL);
          }
          if (a.axis == 1) return launch_tma(k_dht_tma<T, LL, 1, kDhtPlain>, TS::DHT_SMEM, TS::THREADS, tiles, t, s, cls, LL);
          return launch_tma(k_dht_tma<T, LL, 0, kDhtPlain>, TS::DHT_SMEM, TS::THREADS, tiles, t, s, cls, LL);
        }
      }
      break;
    })
  }
  RD_DISPATCH_L(L, {
    constexpr size_t sm = pencil_smem<T, LL>();
    const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
    switch (mode) {
      case kDhtPlain:
        if (a.axis == 2) return launch_pencil(k_dht<T, LL, true, kDhtPlain>, sm, blocks, a, s, kcDhtPlain, LL);
        return launch_pencil(k_dht<T, LL, false, kDhtPlain>, sm, blocks, a, s, kcDhtPlain, LL);
      case kDhtSetup:
        return launch_pencil(k_dht<T, LL, true, kDhtSetup>, sm, blocks, a, s, kcDhtSetup, LL);
      case kDhtUpdate:
        return launch_pencil(k_dht<T, LL, true, kDhtUpdate>, sm, blocks, a, s, kcDhtUpdate, LL);
      case kDhtSym:
        return launch_pencil(k_dht<T, LL, false, kDhtSym>, sm, blocks, a, s, kcDhtSym, LL);
      default:
        return cudaErrorInvalidValue;
    }
  })
}

template <typename T>
cudaError_t Launch<T>::pcg_opx(int L, const PcgOpxArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  const long long npairs = a.g.nn / L / 2;
  if (!tuned_pencil(kcPcgOpx, L) && aligned16(a.w) && aligned16(a.p) && aligned16(a.q) && aligned16(a.kappa) &&
      (!a.x || aligned16(a.x))) {
    RD_DISPATCH_L(L, {
      using TS = TmaRowShape<T, LL>;
      if constexpr (TS::OK) {
        const long long rows = a.g.nn / LL;
        PcgOpxTmaArgs<T> t;
        if (rows % TS::ROWS == 0 && row_map(&t.map_w, a.w, a.g, sizeof(T), TS::ROWS) &&
            row_map(&t.map_k, a.kappa, a.g, sizeof(T), TS::ROWS) && row_map(&t.map_p, a.p, a.g, sizeof(T), TS::ROWS) &&
            (!a.x || row_map(&t.map_x, a.x, a.g, sizeof(T), TS::ROWS))) {
          t.p = a.p;
          t.q = a.q;
          t.x = a.x;
          t.g = a.g;
          t.twA = a.twA;
          t.twB = a.twB;
          t.prm = a.prm;
          t.st = a.st;
          t.fin = a.fin;
          t.rowact = a.rowact;
          return launch_tma(k_pcg_opx_tma<T, LL>, TS::OPX_SMEM, TS::THREADS, rows / TS::ROWS, t, s, kcPcgOpx, LL);
        }
      }
      break;
    })
  }
  RD_DISPATCH_L(L, {
    constexpr size_t sm = pencil_smem<T, LL>();
    const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
    return launch_pencil(k_pcg_opx<T, LL>, sm, blocks, a, s, kcPcgOpx, LL);
  })
}

template <typename T>
cudaError_t Launch<T>::grad(int L, const GradArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  const long long npairs = a.g.nn / L / 2;
  if (a.axis != 2 && !tuned_pencil(kcGrad, L) && !a.q && tma_fits<T>(a.g) && aligned16(a.u0) &&
      (!a.u1 || aligned16(a.u1)) && aligned16(a.w) &&
      aligned16(a.kappa)) {
    RD_DISPATCH_L(L, {
      using TS = TmaShape<T, LL>;
      if constexpr (TS::OK) {
        GradTmaArgs<T> t;
        t.has_u1 = a.u1 ? 1 : 0;
        if (strided_map(&t.map_u0, a.u0, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_u1, a.u1 ? a.u1 : a.u0, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_w, a.w, a.g, sizeof(T), a.axis) &&
            strided_map(&t.map_k, a.kappa, a.g, sizeof(T), a.axis)) {
          t.g = a.g;
          t.twA = a.twA;
          t.twB = a.twB;
          t.fin = a.fin;
          t.tiles = a.tiles;
          t.ntiles_act = a.ntiles_act;
          const long long tiles = (long long)(a.g.n[2] / TS::W) * (a.axis == 1 ? a.g.n[0] : a.g.n[1]);
          if (a.axis == 1) return launch_tma(k_grad_tma<T, LL, 1>, TS::GRAD_SMEM, TS::THREADS, tiles, t, s, kcGrad, LL);
          return launch_tma(k_grad_tma<T, LL, 0>, TS::GRAD_SMEM, TS::THREADS, tiles, t, s, kcGrad, LL);
        }
      }
      break;
    })
  }
  RD_DISPATCH_L(L, {
    constexpr size_t sm = pencil_smem<T, LL>();
    const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
    if (a.axis == 2) return launch_pencil(k_grad<T, LL, true>, sm, blocks, a, s, kcGrad, LL);
    return launch_pencil(k_grad<T, LL, false>, sm, blocks, a, s, kcGrad, LL);
  })
}

template <typename T>
cudaError_t Launch<T>::pw(int kind, const PwArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  const long long blocks = (a.nn + kThreads - 1) / kThreads;
#define RD_PW(K) \
  case K: return launch_pencil(k_pw<T, K>, 0, blocks, a, s, kcPointwise);
  switch (kind) {
    RD_PW(kPwFwdPre)
    RD_PW(kPwFwdPost)
    RD_PW(kPwMisfit)
    RD_PW(kPwAdjPre)
    RD_PW(kPwAdjPost)
    RD_PW(kPwTlPre)
    RD_PW(kPwTlPost)
    RD_PW(kPwNeg)
    RD_PW(kPwState)
    default: return cudaErrorInvalidValue;
  }
#undef RD_PW
}

template <typename T>
cudaError_t Launch<T>::coef(const CoefArgs<T>& a, cudaStream_t s) {
  using namespace detail;
  return launch_pencil(k_coef<T>, 0, (a.nn + kThreads - 1) / kThreads, a, s);
}

template <typename T>
cudaError_t Launch<T>::phi(const PhiArgs<T>& a, cudaStream_t s) {
  const size_t smem = size_t(a.np) * sizeof(double);
  const void* fn = reinterpret_cast<const void*>(k_phi<T>);
  int grid = detail::grid_for(fn, smem, (long long)a.g.n[0] * a.g.n[1]);
  k_phi<T><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::phit(const PhiArgs<T>& a, double* out, double scale, cudaStream_t s) {
  dim3 grid((unsigned)(a.g.n[0] < 64 ? a.g.n[0] : 64), (unsigned)a.np);
  k_phit<T><<<grid, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_phit_sum<T><<<(a.np + 127) / 128, 128, 0, s>>>(a.part, out, a.np, a.g.n[0], scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::from_f64(const double* in, T* out, long long nn, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_convert<T, double>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_convert<T, double><<<grid, kThreads, 0, s>>>(in, out, nn, 1.0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_f64(const T* in, double* out, long long nn, double scale, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_convert<double, T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_convert<double, T><<<grid, kThreads, 0, s>>>(in, out, nn, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::normsq(const NormArgs<T>& a, cudaStream_t s) {
  return detail::launch_pencil(k_normsq<T>, 0, (a.nn + kThreads - 1) / kThreads, a, s, kcPointwise);
}

template <typename T>
cudaError_t Launch<T>::cg_final(T* x, const T* p, const PcgState* st, long long nn, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_cg_final<T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_cg_final<T><<<grid, kThreads, 0, s>>>(x, p, st, nn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::x_init(T* x, const PcgState* st, long long nn, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_x_init<T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_x_init<T><<<grid, kThreads, 0, s>>>(x, st, nn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::guess(T* r, T* x, T* fs, const T* d1, const T* d2, const T* g1, const T* g2, int order,
                             long long nn, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_guess<T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_guess<T><<<grid, kThreads, 0, s>>>(r, x, fs, d1, d2, g1, g2, order, nn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::guess_keep(T* d, T* g, const T* x, const T* r, const T* fs, long long nn, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_guess_keep<T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_guess_keep<T><<<grid, kThreads, 0, s>>>(d, g, x, r, fs, nn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::combine(const T* qk, const T* qr, double ca, double cb, double* out, long long nn,
                               cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_combine<T>);
  int grid = detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads);
  k_combine<T><<<grid, kThreads, 0, s>>>(qk, qr, ca, cb, out, nn);
  return cudaGetLastError();
}

}  // namespace rd
