// TMA-staged pencil passes along the strided axes (0 and 1).
//
// A tile is W columns (64 bytes of adjacent i2 values: 16 FP32 or 8 FP64) by
// the full pencil length L along the pass axis.  cp.async.bulk.tensor moves
// tiles between global and shared memory with the 64-byte swizzle (16-byte
// chunk bits [4:5] of the shared-memory byte offset XOR bits [7:8]), which
// makes the pencil-group reads conflict-free.  The inputs of tile i + 2 are
// prefetched while tile i is computed (two stages); outputs are written back
// into their tile in shared memory and stored with a TMA store.  Every
// mbarrier wait is bounded: on timeout the block records kStTimeout in the
// solver state and exits together.
#pragma once

#include <cuda.h>

#include "rd_passes.cuh"

namespace rd {

constexpr unsigned kWaitLimit = 1u << 26;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Waits for phase `parity` of the barrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = kWaitLimit) {
  const uint32_t a = smem_addr(bar);
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Loads issued on one mbarrier and phases seen completed.  Loads on a
// barrier are issued and awaited in order, so phase k completes with parity
// k & 1.  After a timed-out wait, drain() waits (with the same limit) for the
// loads still in flight, so that no copy lands in shared memory after the
// block has exited.
struct TmaPending {
  unsigned issued = 0, done = 0;
};

__device__ __forceinline__ void drain(uint64_t* bar, const TmaPending& p) {
  for (unsigned k = p.done; k < p.issued; ++k)
    if (!mbar_wait(bar, k & 1)) break;
}

// Two stages used alternately: load k goes to stage k & 1 and completes
// phase k >> 1 of its barrier.  Drains loads done..issued-1.
__device__ __forceinline__ void drain2(uint64_t* full, unsigned done, unsigned issued) {
  for (unsigned k = done; k < issued; ++k)
    if (!mbar_wait(&full[k & 1], (k >> 1) & 1)) break;
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store3(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

// Element-wise add of a shared-memory tile into global memory (the add is
// performed by the memory system; f32 element type from the tensor map).
__device__ __forceinline__ void tma_reduce_add3(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Copy the two twiddle tables of length L into shared memory (whole block).
template <typename T, int L>
__device__ __forceinline__ void stage_twiddles(cpx<T>* dst, const cpx<T>* twA, const cpx<T>* twB) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    dst[i] = ldtw(&twA[i]);
    dst[L + i] = ldtw(&twB[i]);
  }
}

// Tile geometry of the strided-axis TMA kernels.
template <typename T, int L>
struct TmaShape {
  static constexpr int W = 64 / int(sizeof(T));      // columns per tile
  static constexpr int PAIRS = W / 2;                 // pencil pairs per tile
  static constexpr int TH = Shape<L>::TH;
  static constexpr int R = Shape<L>::R;
  static constexpr int THREADS = PAIRS * TH;
  static constexpr int TILE_BYTES = 64 * L;           // one field tile
  static constexpr int XSTRIDE = R * (TH + 1);        // exchange buffer per group (complex)
  static constexpr int XBYTES = PAIRS * XSTRIDE * int(sizeof(cpx<T>));
  static constexpr bool OK = THREADS >= 32;           // whole warps only
  static constexpr int TWBYTES = 2 * L * int(sizeof(cpx<T>));
  static constexpr size_t OP_SMEM = 3 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
  static constexpr size_t OPR_SMEM = 2 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
  static constexpr size_t DHT_SMEM = 2 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
  static constexpr size_t GRAD_SMEM = 3 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
};

// Pair (columns 2g, 2g + 1) of row `row` inside a swizzled 64-byte-row tile.
template <typename T>
__device__ __forceinline__ cpx<T>* tile_pair(unsigned char* tile, int row, int g) {
  uint32_t b = uint32_t(row) * 64u + uint32_t(g) * uint32_t(2 * sizeof(T));
  b ^= (b >> 3) & 0x30u;
  return reinterpret_cast<cpx<T>*>(tile + b);
}

// Tile t of a strided pass -> TMA coordinates {i2, i1, i0} of its corner.
__device__ __forceinline__ void tile_coords(const Geom& g, int axis, int W, long long t, int& c0, int& c1,
                                            int& c2) {
  const int nb = g.n[2] / W;
  const int blk = int(t % nb);
  const int other = int(t / nb);
  c0 = blk * W;
  if (axis == 1) {
    c1 = 0;
    c2 = other;   // i0
  } else {
    c1 = other;   // i1
    c2 = 0;
  }
}

template <typename T>
struct OpTmaArgs {
  CUtensorMap map_u;
  CUtensorMap map_k;
  CUtensorMap map_q;   // accumulator: loaded, updated and stored in place
  double c0;
  int use_kf;
  int reduce;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;
  Fin fin;
  // Optional list of the tiles to process (device; null = every tile) and
  // its length (device).  Tiles where kappa vanishes identically contribute
  // exactly zero to d_axis(kappa d_axis u) and are left out of the list.
  const int* tiles;
  const int* ntiles_act;
};

// q <- q + coef * d_axis(kappa d_axis u), coef = c0 (k_f) s; optionally
// reduces sum kappa (L d_axis u)^2, this axis's share of (u, (I - sA) u).
//
// Shared memory holds one tile each of u, kappa and q plus the FFT exchange
// area.  Each input of tile i + 1 is requested as soon as this block has
// taken the corresponding values of tile i into registers (u before the
// first transform, kappa before the second, q after its store was read), so
// the loads overlap the transforms while three blocks fit on an SM.
template <typename T, int L, int AXIS>
__global__ void __launch_bounds__(TmaShape<T, L>::THREADS) k_op_tma(const __grid_constant__ OpTmaArgs<T> a) {
  using S = TmaShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* u_buf = smem;
  unsigned char* k_buf = smem + TB;
  unsigned char* q_buf = smem + 2 * TB;
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 3 * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 3 * TB + S::XBYTES);
  const cpx<T>* twA = tws;
  const cpx<T>* twB = tws + L;
  stage_twiddles<T, L>(tws, a.twA, a.twB);
  __shared__ uint64_t ubar, kbar, qbar;
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles =
      a.tiles ? (long long)*a.ntiles_act : (long long)(a.g.n[2] / S::W) * (AXIS == 1 ? a.g.n[0] : a.g.n[1]);
  auto tile_at = [&](long long j) { return a.tiles ? (long long)a.tiles[j] : j; };
  const T coef = T(a.c0 * (a.use_kf ? a.prm->k_f : 1.0) * a.prm->s / (double(L) * double(L)));

  TmaPending pu, pk, pq;
  auto issue = [&](unsigned char* dst, const CUtensorMap* map, uint64_t* bar, TmaPending& pd, long long tile) {
    int c0, c1, c2;
    tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
    mbar_expect_tx(bar, TB);
    tma_load3(dst, map, c0, c1, c2, bar);
    ++pd.issued;
  };

  if (threadIdx.x == 0) {
    mbar_init(&ubar, 1);
    mbar_init(&kbar, 1);
    mbar_init(&qbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0 && t0 < ntiles) {
    issue(u_buf, &a.map_u, &ubar, pu, tile_at(t0));
    issue(k_buf, &a.map_k, &kbar, pk, tile_at(t0));
    issue(q_buf, &a.map_q, &qbar, pq, tile_at(t0));
  }
  double red = 0.0;
  bool bad = false;
  int i = 0;
  for (long long j = t0; j < ntiles; j += stride, ++i) {
    const long long tile = tile_at(j);
    const bool more = j + stride < ntiles;
    bool ok = mbar_wait(&ubar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pu.done;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = *tile_pair<T>(u_buf, idx_a<L>(r, t), g);
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every u value is in registers
    if (threadIdx.x == 0) {
      if (more) issue(u_buf, &a.map_u, &ubar, pu, tile_at(j + stride));
      if (i > 0) {
        // q_buf is free once the previous tile's store has read it
        bulk_wait_read0();
        issue(q_buf, &a.map_q, &qbar, pq, tile);
      }
    }
    fft_ab<T, L, -1, kTwShared>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(v, sm, t, twB);
    ok = mbar_wait(&kbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pk.done;
    T loc = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T> k = *tile_pair<T>(k_buf, idx_a<L>(r, t), g);
      if (a.reduce) loc += k.x * v[r].x * v[r].x + k.y * v[r].y * v[r].y;
      v[r].x *= k.x;
      v[r].y *= k.y;
    }
    red += double(loc);
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every kappa value is in registers
    if (threadIdx.x == 0 && more) issue(k_buf, &a.map_k, &kbar, pk, tile_at(j + stride));
    fft_ab<T, L, -1, kTwShared>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(v, sm, t, twB);
    ok = mbar_wait(&qbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pq.done;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T>* qp = tile_pair<T>(q_buf, idx_a<L>(r, t), g);
      cpx<T> q = *qp;
      q.x += coef * v[r].x;
      q.y += coef * v[r].y;
      *qp = q;
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      int c0, c1, c2;
      tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
      tma_store3(&a.map_q, q_buf, c0, c1, c2);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
  if (bad) {
    if (threadIdx.x == 0) {
      a.st->status = kStTimeout;
      a.st->sticky = kStTimeout;
      drain(&ubar, pu);
      drain(&kbar, pk);
      drain(&qbar, pq);
    }
    return;
  }
  if (a.reduce) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

// The same operator pass with the accumulation done by a TMA reduce-add
// into q (FP32 fields): q is never loaded into the block, and the kappa
// tile, once its values are in registers, stages coef * d(kappa d u) for
// the reduction.  Two tiles plus the exchange area per block.  Each element
// of q receives exactly one add per pass, so the result is deterministic.
template <typename T, int L, int AXIS>
__global__ void __launch_bounds__(TmaShape<T, L>::THREADS) k_op_tma_red(const __grid_constant__ OpTmaArgs<T> a) {
  static_assert(sizeof(T) == 4, "the tensor reduce-add is used for FP32 fields");
  using S = TmaShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* u_buf = smem;
  unsigned char* k_buf = smem + TB;   // kappa, then the tile added into q
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 2 * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 2 * TB + S::XBYTES);
  const cpx<T>* twA = tws;
  const cpx<T>* twB = tws + L;
  stage_twiddles<T, L>(tws, a.twA, a.twB);
  __shared__ uint64_t ubar, kbar;
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles =
      a.tiles ? (long long)*a.ntiles_act : (long long)(a.g.n[2] / S::W) * (AXIS == 1 ? a.g.n[0] : a.g.n[1]);
  auto tile_at = [&](long long j) { return a.tiles ? (long long)a.tiles[j] : j; };
  const T coef = T(a.c0 * (a.use_kf ? a.prm->k_f : 1.0) * a.prm->s / (double(L) * double(L)));
  TmaPending pu, pk;
  auto issue = [&](unsigned char* dst, const CUtensorMap* map, uint64_t* bar, TmaPending& pd, long long tile) {
    int c0, c1, c2;
    tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
    mbar_expect_tx(bar, TB);
    tma_load3(dst, map, c0, c1, c2, bar);
    ++pd.issued;
  };
  if (threadIdx.x == 0) {
    mbar_init(&ubar, 1);
    mbar_init(&kbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0 && t0 < ntiles) {
    issue(u_buf, &a.map_u, &ubar, pu, tile_at(t0));
    issue(k_buf, &a.map_k, &kbar, pk, tile_at(t0));
  }
  double red = 0.0;
  bool bad = false;
  int i = 0;
  for (long long j = t0; j < ntiles; j += stride, ++i) {
    const long long tile = tile_at(j);
    const bool more = j + stride < ntiles;
    bool ok = mbar_wait(&ubar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pu.done;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = *tile_pair<T>(u_buf, idx_a<L>(r, t), g);
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every u value is in registers
    if (threadIdx.x == 0) {
      if (more) issue(u_buf, &a.map_u, &ubar, pu, tile_at(j + stride));
      if (i > 0) {
        // kappa of this tile goes into k_buf once the previous tile's
        // reduce-add has read it; requested here, two transforms before it
        // is needed, so that no warp waits for that read at a block barrier
        bulk_wait_read0();
        issue(k_buf, &a.map_k, &kbar, pk, tile);
      }
    }
    fft_ab<T, L, -1, kTwShared>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(v, sm, t, twB);
    ok = mbar_wait(&kbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pk.done;
    T loc = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T> k = *tile_pair<T>(k_buf, idx_a<L>(r, t), g);
      if (a.reduce) loc += k.x * v[r].x * v[r].x + k.y * v[r].y * v[r].y;
      v[r].x *= k.x;
      v[r].y *= k.y;
    }
    red += double(loc);
    __syncthreads();   // every kappa value is in registers: k_buf is free
    fft_ab<T, L, -1, kTwShared>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(v, sm, t, twB);
#pragma unroll
    for (int r = 0; r < R; ++r) *tile_pair<T>(k_buf, idx_a<L>(r, t), g) = {coef * v[r].x, coef * v[r].y};
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      int c0, c1, c2;
      tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
      tma_reduce_add3(&a.map_q, k_buf, c0, c1, c2);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
  if (bad) {
    if (threadIdx.x == 0) {
      a.st->status = kStTimeout;
      a.st->sticky = kStTimeout;
      drain(&ubar, pu);
      drain(&kbar, pk);
    }
    return;
  }
  if (a.reduce) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

template <typename T>
struct DhtTmaArgs {
  CUtensorMap map_in;
  CUtensorMap map_out;
  int axis;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;
  Fin fin;
};

// Hartley pass along a strided axis: MODE kDhtPlain (out = H in, written at
// layout-B positions of each pencil) or kDhtSym (out = H S' H in, rz reduced).
template <typename T, int L, int AXIS, int MODE>
__global__ void __launch_bounds__(TmaShape<T, L>::THREADS, (MODE == kDhtSym && sizeof(T) == 4) ? 4 : 1) k_dht_tma(const __grid_constant__ DhtTmaArgs<T> a) {
  using S = TmaShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto st_buf = [&](int b) { return smem + b * TB; };
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 2 * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 2 * TB + S::XBYTES);
  const cpx<T>* twA = tws;
  const cpx<T>* twB = tws + L;
  stage_twiddles<T, L>(tws, a.twA, a.twB);
  __shared__ uint64_t full[2];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles = (long long)(a.g.n[2] / S::W) * (AXIS == 1 ? a.g.n[0] : a.g.n[1]);
  double symc = 0.0, inv_nn = 0.0;
  if (MODE == kDhtSym) {
    symc = a.prm->s * a.prm->k_f * a.prm->kbar1;
    inv_nn = a.prm->inv_nn;
  }
  unsigned issued = 0;
  auto issue = [&](long long tile, int b) {
    int c0, c1, c2;
    tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
    mbar_expect_tx(&full[b], TB);
    tma_load3(st_buf(b), &a.map_in, c0, c1, c2, &full[b]);
    ++issued;
  };
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0) {
    if (t0 < ntiles) issue(t0, 0);
    if (t0 + stride < ntiles) issue(t0 + stride, 1);
  }
  double red = 0.0;
  bool bad = false;
  int i = 0;
  for (long long tile = t0; tile < ntiles; tile += stride, ++i) {
    const int b = i & 1;
    bool ok = mbar_wait(&full[b], (i >> 1) & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = *tile_pair<T>(st_buf(b), idx_a<L>(r, t), g);
    if (threadIdx.x == 0 && i > 0 && tile + stride < ntiles) {
      // the other stage is free once the previous tile's store has read it
      bulk_wait_read0();
      issue(tile + stride, b ^ 1);
    }
    fft_ab<T, L, -1, kTwShared>(v, sm, t, twA);
    if (MODE != kDhtSym) hartley_combine<T, L, true>(v, t);
    T loc = T(0);
    if (MODE == kDhtSym) {
      int c0, c1, c2;
      tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
      const int i1 = c1, i2 = c0 + 2 * g;
      const int k1 = kwave_rt(i1, a.g.n[1]), k2a = kwave_rt(i2, a.g.n[2]), k2b = kwave_rt(i2 + 1, a.g.n[2]);
      const T base_a = T(k1 * k1 + k2a * k2a);
      const T base_b = T(k1 * k1 + k2b * k2b);
      loc = sym_apply<T, L>(v, t, base_a, base_b, T(symc), T(inv_nn));
      fft_ba<T, L, +1, kTwShared>(v, sm, t, twB);
#pragma unroll
      for (int r = 0; r < R; ++r) *tile_pair<T>(st_buf(b), idx_a<L>(r, t), g) = v[r];
    } else {
      // the input values of this pencil were read before the exchange; the
      // whole group has passed a __syncwarp since, so writing in place is safe
#pragma unroll
      for (int r = 0; r < R; ++r) *tile_pair<T>(st_buf(b), idx_b<L>(r, t), g) = v[r];
    }
    red += double(loc);
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      int c0, c1, c2;
      tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
      tma_store3(&a.map_out, st_buf(b), c0, c1, c2);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
  if (bad) {
    if (threadIdx.x == 0) {
      a.st->status = kStTimeout;
      a.st->sticky = kStTimeout;
      drain2(full, unsigned(i), issued);
    }
    return;
  }
  if (MODE == kDhtSym) {
    double vv[1] = {red};
    reduce_finish<1>(vv, a.fin);
  }
}

template <typename T>
struct GradTmaArgs {
  CUtensorMap map_u0;
  CUtensorMap map_u1;   // equal to map_u0 when has_u1 == 0
  CUtensorMap map_w;
  CUtensorMap map_k;
  int has_u1;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Fin fin;
  const int* tiles;        // as in OpTmaArgs: tiles where kappa is not zero
  const int* ntiles_act;
};

// Gradient pass along a strided axis (the reduction of k_grad without the
// per-voxel output): sum_x kappa1 d_axis(u0 + u1) d_axis(w).  Three tile
// buffers: A holds u0 and then kappa, B holds u1, C holds w.  kappa and the
// next u1 are requested as soon as u0 + u1 is in registers, the next w once
// w is, and the next u0 once kappa is, so every load overlaps a transform.
template <typename T, int L, int AXIS>
__global__ void __launch_bounds__(TmaShape<T, L>::THREADS) k_grad_tma(const __grid_constant__ GradTmaArgs<T> a) {
  using S = TmaShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_buf = smem;
  unsigned char* b_buf = smem + TB;
  unsigned char* c_buf = smem + 2 * TB;
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 3 * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 3 * TB + S::XBYTES);
  const cpx<T>* twA = tws;
  const cpx<T>* twB = tws + L;
  stage_twiddles<T, L>(tws, a.twA, a.twB);
  __shared__ uint64_t abar, bbar, cbar;
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles =
      a.tiles ? (long long)*a.ntiles_act : (long long)(a.g.n[2] / S::W) * (AXIS == 1 ? a.g.n[0] : a.g.n[1]);
  auto tile_at = [&](long long j) { return a.tiles ? (long long)a.tiles[j] : j; };
  const T scale = T(1.0 / (double(L) * double(L)));
  const bool two = a.has_u1 != 0;
  TmaPending pa, pb, pc;
  auto issue = [&](unsigned char* dst, const CUtensorMap* map, uint64_t* bar, TmaPending& pd, long long tile) {
    int c0, c1, c2;
    tile_coords(a.g, AXIS, S::W, tile, c0, c1, c2);
    mbar_expect_tx(bar, TB);
    tma_load3(dst, map, c0, c1, c2, bar);
    ++pd.issued;
  };
  if (threadIdx.x == 0) {
    mbar_init(&abar, 1);
    mbar_init(&bbar, 1);
    mbar_init(&cbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0 && t0 < ntiles) {
    issue(a_buf, &a.map_u0, &abar, pa, tile_at(t0));
    if (two) issue(b_buf, &a.map_u1, &bbar, pb, tile_at(t0));
    issue(c_buf, &a.map_w, &cbar, pc, tile_at(t0));
  }
  double red = 0.0;
  bool bad = false;
  int i = 0;
  for (long long j = t0; j < ntiles; j += stride, ++i) {
    const long long tile = tile_at(j);
    const bool more = j + stride < ntiles;
    // u0 is load 2i of barrier A (parity 0), kappa load 2i + 1 (parity 1)
    bool ok = mbar_wait(&abar, 0);
    if (two) ok = ok && mbar_wait(&bbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pa.done;
    if (two) ++pb.done;
    cpx<T> du[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      du[r] = *tile_pair<T>(a_buf, idx_a<L>(r, t), g);
      if (two) du[r] = du[r] + *tile_pair<T>(b_buf, idx_a<L>(r, t), g);
    }
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every u0 and u1 value is in registers
    if (threadIdx.x == 0) {
      issue(a_buf, &a.map_k, &abar, pa, tile);
      if (two && more) issue(b_buf, &a.map_u1, &bbar, pb, tile_at(j + stride));
    }
    fft_ab<T, L, -1, kTwShared>(du, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) du[r] = times_ik(du[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(du, sm, t, twB);
    ok = mbar_wait(&cbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pc.done;
    cpx<T> dw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dw[r] = *tile_pair<T>(c_buf, idx_a<L>(r, t), g);
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every w value is in registers
    if (threadIdx.x == 0 && more) issue(c_buf, &a.map_w, &cbar, pc, tile_at(j + stride));
    fft_ab<T, L, -1, kTwShared>(dw, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) dw[r] = times_ik(dw[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwShared>(dw, sm, t, twB);
    ok = mbar_wait(&abar, 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pa.done;
    T loc = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const cpx<T> k = *tile_pair<T>(a_buf, idx_a<L>(r, t), g);
      loc += k.x * du[r].x * dw[r].x + k.y * du[r].y * dw[r].y;
    }
    red += double(loc * scale);
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every kappa value is in registers
    if (threadIdx.x == 0 && more) issue(a_buf, &a.map_u0, &abar, pa, tile_at(j + stride));
  }
  if (bad) {
    if (threadIdx.x == 0) {
      a.fin.st->status = kStTimeout;
      a.fin.st->sticky = kStTimeout;
      drain(&abar, pa);
      drain(&bbar, pb);
      drain(&cbar, pc);
    }
    return;
  }
  double vv[1] = {red};
  reduce_finish<1>(vv, a.fin);
}

}  // namespace rd

namespace rd {

// ------------------------------------------------ contiguous axis (axis 2)
// A tile is ROWS whole x-pencils (rows of the [n0 n1][n2] view) loaded with
// a 2D tensor map, box {L, ROWS}, no swizzle.  Element (row, i) of a tile
// sits at byte (row L + i) sizeof(T).
template <typename T, int L>
struct TmaRowShape {
  static constexpr int TH = Shape<L>::TH;
  static constexpr int R = Shape<L>::R;
  static constexpr int BASE = (sizeof(T) == 4) ? 4 : 2;
  static constexpr int PAIRS = (32 / TH > BASE) ? 32 / TH : BASE;
  static constexpr int ROWS = 2 * PAIRS;
  static constexpr int THREADS = PAIRS * TH;
  static constexpr int TILE_BYTES = ROWS * L * int(sizeof(T));
  static constexpr int XSTRIDE = R * (TH + 1);
  static constexpr int XBYTES = PAIRS * XSTRIDE * int(sizeof(cpx<T>));
  static constexpr bool OK = (THREADS >= 32) && (THREADS % 32 == 0);
  static constexpr int TWBYTES = 0;   // twiddles are read from global memory (kTwGlobal)
  static constexpr size_t OPX_SMEM = 2 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 128;
  static constexpr size_t OPROW_SMEM = 2 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 128;
  static constexpr size_t UPD_SMEM = 4 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
  static constexpr size_t SETUP_SMEM = 2 * size_t(TILE_BYTES) + XBYTES + TWBYTES + 1024;
};

template <typename T, int L>
__device__ __forceinline__ T* row_elem(unsigned char* tile, int row, int i) {
  return reinterpret_cast<T*>(tile) + row * L + i;
}

__device__ __forceinline__ void tma_load2(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store2(const CUtensorMap* map, const void* src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(c0), "r"(c1)
               : "memory");
}

template <typename T>
struct OpRowTmaArgs {
  CUtensorMap map_u;
  CUtensorMap map_k;
  T* out;
  double c0;
  int use_kf;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;   // timeout flag
};

// out = c0 (k_f) s d_2(kappa d_2 u): the contiguous-axis pass that starts an
// operator application (nothing accumulated, nothing reduced).  u and kappa
// arrive as TMA row tiles, each requested for the next tile as soon as its
// values are in registers; out leaves from registers in layout A, where the
// TH lanes of a group hold TH consecutive elements of a row (coalesced).
template <typename T, int L>
__global__ void __launch_bounds__(TmaRowShape<T, L>::THREADS) k_op_row_tma(const __grid_constant__ OpRowTmaArgs<T> a) {
  using S = TmaRowShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  unsigned char* u_buf = smem;
  unsigned char* k_buf = smem + TB;
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 2 * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 2 * TB + S::XBYTES);
  const cpx<T>* twA = a.twA;   // read through L1 (kTwGlobal)
  const cpx<T>* twB = a.twB;
  (void)tws;
  __shared__ uint64_t ubar, kbar;
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles = a.g.nn / L / S::ROWS;
  const T coef = T(a.c0 * (a.use_kf ? a.prm->k_f : 1.0) * a.prm->s / (double(L) * double(L)));
  TmaPending pu, pk;
  auto issue = [&](unsigned char* dst, const CUtensorMap* map, uint64_t* bar, TmaPending& pd, long long tile) {
    mbar_expect_tx(bar, TB);
    tma_load2(dst, map, 0, int(tile * S::ROWS), bar);
    ++pd.issued;
  };
  if (threadIdx.x == 0) {
    mbar_init(&ubar, 1);
    mbar_init(&kbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0 && t0 < ntiles) {
    issue(u_buf, &a.map_u, &ubar, pu, t0);
    issue(k_buf, &a.map_k, &kbar, pk, t0);
  }
  bool bad = false;
  int i = 0;
  const int ra = 2 * g, rb = 2 * g + 1;
  for (long long tile = t0; tile < ntiles; tile += stride, ++i) {
    const bool more = tile + stride < ntiles;
    T* orow_a = a.out + (tile * S::ROWS + ra) * L;
    T* orow_b = a.out + (tile * S::ROWS + rb) * L;
    bool ok = mbar_wait(&ubar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pu.done;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_a<L>(r, t);
      v[r] = {*row_elem<T, L>(u_buf, ra, n), *row_elem<T, L>(u_buf, rb, n)};
    }
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every u value is in registers
    if (threadIdx.x == 0 && more) issue(u_buf, &a.map_u, &ubar, pu, tile + stride);
    fft_ab<T, L, -1, kTwGlobal>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwGlobal>(v, sm, t, twB);
    ok = mbar_wait(&kbar, i & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pk.done;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_a<L>(r, t);
      v[r].x *= *row_elem<T, L>(k_buf, ra, n);
      v[r].y *= *row_elem<T, L>(k_buf, rb, n);
    }
    fence_proxy_async();   // the reads above come before the next copy into this buffer
    __syncthreads();   // every kappa value is in registers
    if (threadIdx.x == 0 && more) issue(k_buf, &a.map_k, &kbar, pk, tile + stride);
    fft_ab<T, L, -1, kTwGlobal>(v, sm, t, twA);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_b<L>(r, t)));
    fft_ba<T, L, +1, kTwGlobal>(v, sm, t, twB);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_a<L>(r, t);
      orow_a[n] = coef * v[r].x;
      orow_b[n] = coef * v[r].y;
    }
  }
  if (bad && threadIdx.x == 0) {
    a.st->status = kStTimeout;
    a.st->sticky = kStTimeout;
    drain(&ubar, pu);
    drain(&kbar, pk);
  }
}

template <typename T>
struct PcgOpxTmaArgs {
  CUtensorMap map_w;
  CUtensorMap map_k;
  CUtensorMap map_p;
  CUtensorMap map_x;
  T* p;          // p is read through map_p and rewritten in place
  T* q;
  T* x;          // CG iterate: the deferred x += alpha p (see PcgOpxArgs; null: none)
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  Params* prm;
  PcgState* st;
  Fin fin;   // reduces |p|^2 and sum kappa (L d_2 p)^2 (kFinPqAdd)
  // Optional flag per row tile (device; null = all set): 0 when kappa
  // vanishes on every row of the tile, where q = p exactly and the
  // operator's transforms are skipped.
  const int* rowact;
};

// z = H_2(w); p = z + beta p; q = p - s k_f d_2(kappa d_2 p)  (fields written
// at layout-B positions of each pencil); reduces |p|^2 and sum kappa
// (L d_2 p)^2.  Two tile buffers, each holding two fields in turn: w, then
// the x of the deferred update (buffer 0); the old p, then kappa (buffer 1).
// w is in registers before x is needed, and p before kappa, so every load
// is issued as soon as its buffer is free: x while the Hartley pass runs,
// kappa and the next w after it, the next p once kappa is in registers.
// Two buffers instead of four leave room for more blocks per SM.  The new p
// and q leave from registers: in layout B the TH lanes of a group hold TH
// consecutive elements of a row per register, so the stores are coalesced.
// q = p + ... takes p from a register copy when that copy is small, else
// re-reads the value this thread has just stored.
template <typename T, int L>
__global__ void __launch_bounds__(TmaRowShape<T, L>::THREADS) k_pcg_opx_tma(const __grid_constant__ PcgOpxTmaArgs<T> a) {
  using S = TmaRowShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  unsigned char* buf0 = smem;        // w, then x
  unsigned char* buf1 = smem + TB;   // old p, then kappa
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 2 * TB);
  const cpx<T>* twA = a.twA;   // read through L1 (kTwGlobal)
  const cpx<T>* twB = a.twB;
  __shared__ uint64_t wbar, xbar, pbar, kbar;
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles = a.g.nn / L / S::ROWS;
  const double betad = a.st->beta;
  // from the second iteration on (st->it counts completed iterations) the
  // old p also serves the deferred x += alpha p of the previous iteration
  const bool xupd = a.x && a.st->it > 0;
  const bool use_p = (betad != 0.0) || xupd;
  const T beta = T(betad);
  const T alpha = xupd ? T(a.st->alpha) : T(0);
  const T coef = T(-a.prm->s * a.prm->k_f / (double(L) * double(L)));
  TmaPending pw, px, pp, pk;
  auto issue = [&](unsigned char* dst, const CUtensorMap* map, uint64_t* bar, TmaPending& pd, long long tile) {
    mbar_expect_tx(bar, TB);
    tma_load2(dst, map, 0, int(tile * S::ROWS), bar);
    ++pd.issued;
  };
  if (threadIdx.x == 0) {
    mbar_init(&wbar, 1);
    mbar_init(&xbar, 1);
    mbar_init(&pbar, 1);
    mbar_init(&kbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0 && t0 < ntiles) {
    issue(buf0, &a.map_w, &wbar, pw, t0);
    if (use_p) issue(buf1, &a.map_p, &pbar, pp, t0);
  }
  bool bad = false;
  double red_pp = 0.0, red_k = 0.0;
  const int ra = 2 * g, rb = 2 * g + 1;
  for (long long tile = t0; tile < ntiles; tile += stride) {
    const bool more = tile + stride < ntiles;
    const bool act = !a.rowact || a.rowact[tile] != 0;
    T* prow_a = a.p + (tile * S::ROWS + ra) * L;
    T* prow_b = a.p + (tile * S::ROWS + rb) * L;
    T* qrow_a = a.q + (tile * S::ROWS + ra) * L;
    T* qrow_b = a.q + (tile * S::ROWS + rb) * L;
    bool ok = mbar_wait(&wbar, pw.done & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    ++pw.done;
    cpx<T> v[R];
    T lpp = T(0), lk = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_a<L>(r, t);
      v[r] = {*row_elem<T, L>(buf0, ra, n), *row_elem<T, L>(buf0, rb, n)};
    }
    // every w value is in registers: buffer 0 takes x (the proxy fence
    // orders these shared-memory reads before the copy engine's write)
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0 && xupd) issue(buf0, &a.map_x, &xbar, px, tile);
    constexpr bool KEEP_P = R * int(sizeof(T)) <= 64;
    cpx<T> pv[KEEP_P ? R : 1];
    // Five transforms per tile through two copies of the transform code (a
    // loop that is not unrolled keeps the kernel within the instruction
    // cache): step 0 is the Hartley pass of w (forward, A -> B); steps 1-4
    // are d(kappa d p): forward B -> A, i k, inverse A -> B, kappa, forward
    // B -> A, i k, inverse A -> B.  The inverse A -> B transform is the
    // forward one between two conjugations.  Row tiles without kappa stop
    // after step 0 (q = p there).
    const int nsteps = act ? 5 : 1;
#pragma unroll 1
    for (int step = 0; step < nsteps; ++step) {
      if ((step & 1) == 0) {
        if (step > 0) conj_all<T, R>(v);
        fft_ab<T, L, -1, kTwGlobal>(v, sm, t, twA);
        if (step > 0) conj_all<T, R>(v);
      } else {
        fft_ba<T, L, -1, kTwGlobal>(v, sm, t, twB);
      }
      if (step == 0) {
        hartley_combine<T, L, true>(v, t);
        if (use_p) {
          ok = mbar_wait(&pbar, pp.done & 1);
          if (ok && xupd) ok = mbar_wait(&xbar, px.done & 1);
          if (__syncthreads_or(!ok)) { bad = true; break; }
          ++pp.done;
          if (xupd) ++px.done;
          T* xrow_a = xupd ? a.x + (tile * S::ROWS + ra) * L : nullptr;
          T* xrow_b = xupd ? a.x + (tile * S::ROWS + rb) * L : nullptr;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = idx_b<L>(r, t);
            const T pa = *row_elem<T, L>(buf1, ra, n), pb = *row_elem<T, L>(buf1, rb, n);
            v[r].x += beta * pa;
            v[r].y += beta * pb;
            if (xupd) {
              xrow_a[n] = *row_elem<T, L>(buf0, ra, n) + alpha * pa;
              xrow_b[n] = *row_elem<T, L>(buf0, rb, n) + alpha * pb;
            }
          }
          fence_proxy_async();
          __syncthreads();   // every old p and x value is in registers: both buffers are free
        }
        if (threadIdx.x == 0) {
          if (act)
            issue(buf1, &a.map_k, &kbar, pk, tile);
          else if (use_p && more)
            issue(buf1, &a.map_p, &pbar, pp, tile + stride);
          if (more) issue(buf0, &a.map_w, &wbar, pw, tile + stride);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = idx_b<L>(r, t);
          if constexpr (KEEP_P) pv[r] = v[r];
          lpp += v[r].x * v[r].x + v[r].y * v[r].y;
          prow_a[n] = v[r].x;
          prow_b[n] = v[r].y;
        }
      } else if (step & 1) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = times_ik(v[r], kwave<L>(idx_a<L>(r, t)));
      } else if (step == 2) {
        ok = mbar_wait(&kbar, pk.done & 1);
        if (__syncthreads_or(!ok)) { bad = true; break; }
        ++pk.done;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = idx_b<L>(r, t);
          const T ka = *row_elem<T, L>(buf1, ra, n), kb = *row_elem<T, L>(buf1, rb, n);
          lk += ka * v[r].x * v[r].x + kb * v[r].y * v[r].y;
          v[r].x *= ka;
          v[r].y *= kb;
        }
        fence_proxy_async();
        __syncthreads();   // every kappa value is in registers: buffer 1 takes the next p
        if (threadIdx.x == 0 && use_p && more) issue(buf1, &a.map_p, &pbar, pp, tile + stride);
      }
    }
    if (bad) break;
    red_pp += double(lpp);
    red_k += double(lk);
    if (!act) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = {T(0), T(0)};
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_b<L>(r, t);
      if constexpr (KEEP_P) {
        qrow_a[n] = pv[r].x + coef * v[r].x;
        qrow_b[n] = pv[r].y + coef * v[r].y;
      } else {
        qrow_a[n] = prow_a[n] + coef * v[r].x;
        qrow_b[n] = prow_b[n] + coef * v[r].y;
      }
    }
  }
  if (bad) {
    if (threadIdx.x == 0) {
      a.st->status = kStTimeout;
      a.st->sticky = kStTimeout;
      drain(&wbar, pw);
      drain(&xbar, px);
      drain(&pbar, pp);
      drain(&kbar, pk);
    }
    return;
  }
  double vv[2] = {red_pp, red_k};
  reduce_finish<2>(vv, a.fin);
}

template <typename T>
struct DhtRowTmaArgs {
  CUtensorMap map_r;
  CUtensorMap map_q;
  CUtensorMap map_out;
  Geom g;
  const cpx<T>* twA;
  const cpx<T>* twB;
  PcgState* st;
  Fin fin;
};

// Setup: ff = ||r||^2, out = H_2(r).
// Update: r -= alpha q, rr = ||r||^2, out = H_2(r) (the iterate's x += alpha p
// is deferred to the next iteration's first Hartley pass, see DhtArgs).
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(TmaRowShape<T, L>::THREADS) k_dht_row_tma(const __grid_constant__ DhtRowTmaArgs<T> a) {
  using S = TmaRowShape<T, L>;
  constexpr int R = S::R, TH = S::TH, TB = S::TILE_BYTES;
  constexpr int NF = (MODE == kDhtUpdate) ? 2 : 1;   // fields per stage: r (, q)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage b: r at smem + (b NF + 0) TB, q at +1
  auto fld = [&](int b, int f) { return smem + (b * NF + f) * TB; };
  cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem + 2 * NF * TB);
  cpx<T>* tws = reinterpret_cast<cpx<T>*>(smem + 2 * NF * TB + S::XBYTES);
  const cpx<T>* twA = a.twA;   // read through L1 (kTwGlobal)
  const cpx<T>* twB = a.twB;
  (void)tws;
  __shared__ uint64_t full[2];
  const int g = threadIdx.x / TH, t = threadIdx.x % TH;
  cpx<T>* sm = xbuf + g * S::XSTRIDE;
  const long long ntiles = a.g.nn / L / S::ROWS;
  const T alpha = (MODE == kDhtUpdate) ? T(a.st->alpha) : T(0);
  unsigned issued = 0;
  auto issue = [&](long long tile, int b) {
    const int row0 = int(tile * S::ROWS);
    ++issued;
    mbar_expect_tx(&full[b], NF * TB);
    tma_load2(fld(b, 0), &a.map_r, 0, row0, &full[b]);
    if (MODE == kDhtUpdate) tma_load2(fld(b, 1), &a.map_q, 0, row0, &full[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const long long t0 = blockIdx.x, stride = gridDim.x;
  if (threadIdx.x == 0) {
    if (t0 < ntiles) issue(t0, 0);
    if (t0 + stride < ntiles) issue(t0 + stride, 1);
  }
  bool bad = false;
  double red = 0.0;
  int i = 0;
  const int ra = 2 * g, rb = 2 * g + 1;
  for (long long tile = t0; tile < ntiles; tile += stride, ++i) {
    const int b = i & 1;
    bool ok = mbar_wait(&full[b], (i >> 1) & 1);
    if (__syncthreads_or(!ok)) { bad = true; break; }
    cpx<T> v[R];
    T loc = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_a<L>(r, t);
      T* r0 = row_elem<T, L>(fld(b, 0), ra, n);
      T* r1 = row_elem<T, L>(fld(b, 0), rb, n);
      cpx<T> rv = {*r0, *r1};
      if (MODE == kDhtUpdate) {
        const T q0 = *row_elem<T, L>(fld(b, 1), ra, n), q1 = *row_elem<T, L>(fld(b, 1), rb, n);
        rv.x -= alpha * q0;
        rv.y -= alpha * q1;
        *r0 = rv.x;
        *r1 = rv.y;
      }
      loc += rv.x * rv.x + rv.y * rv.y;
      v[r] = rv;
    }
    red += double(loc);
    if (threadIdx.x == 0 && i > 0 && tile + stride < ntiles) {
      // the other stage is free once the previous tile's stores have read it
      bulk_wait_read0();
      issue(tile + stride, b ^ 1);
    }
    fft_ab<T, L, -1, kTwGlobal>(v, sm, t, twA);
    hartley_combine<T, L, true>(v, t);
    // Hartley values go to the q tile (update) or back into the r tile (setup);
    // this group's q values were read before the exchange's __syncwarp
    unsigned char* ob = (MODE == kDhtUpdate) ? fld(b, 1) : fld(b, 0);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = idx_b<L>(r, t);
      *row_elem<T, L>(ob, ra, n) = v[r].x;
      *row_elem<T, L>(ob, rb, n) = v[r].y;
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int row0 = int(tile * S::ROWS);
      if (MODE == kDhtUpdate) tma_store2(&a.map_r, fld(b, 0), 0, row0);
      tma_store2(&a.map_out, ob, 0, row0);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait0();
  if (bad) {
    if (threadIdx.x == 0) {
      a.st->status = kStTimeout;
      a.st->sticky = kStTimeout;
      drain2(full, unsigned(i), issued);
    }
    return;
  }
  double vv[1] = {red};
  reduce_finish<1>(vv, a.fin);
}

}  // namespace rd
