// Host orchestration of the reaction-diffusion solve and the C ABI of
// include/rd.h.
//
// One time step (Sec. 3.3, Strang splitting, read as L(tau/2) CN(tau)
// L(tau/2)):
//   c*  = L_s(c_n)                      s = tau/2, exact logistic flow
//   c** = c* + dx,  (I - s A) dx = 2 s A c*      (Crank-Nicolson increment)
//   c_{n+1} = L_s(c**)
// The adjoint sweep is the exact transpose of this step (the CN matrix is
// symmetric; the logistic step transposes to multiplication by dL_s/dc),
// with alpha(1) = d - c(1) (Eq. tumor:adj-final) and the parameter
// gradients of Eq. tumor:inv / tumor:inv_diff accumulated on the way back.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/rd.h"
#include "rd_launch.cuh"
#include "rd_tables.h"

namespace rd {

bool supported_length(int L) {
  return L == 8 || L == 16 || L == 32 || L == 64 || L == 96 || L == 128 || L == 256;
}

// ------------------------------------------------------- launch timing
namespace {
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  double ms[kcCount] = {};
  long long count[kcCount] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& r : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.cls] += t;
        count[r.cls] += 1;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
};
Profiler& prof() {
  static Profiler p;
  return p;
}
const char* kClassNames[kcCount] = {"op_axis2",   "op_axis01",  "pcg_opx", "dht_setup", "dht_plain",
                                    "dht_update", "dht_sym",    "grad",    "pointwise", "other"};
}  // namespace

namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
struct MapKey {
  uintptr_t p;
  int n0, n1, n2, esz, kind;   // kind: 0/1 strided axis, 100 + rows for row maps
  bool operator<(const MapKey& o) const {
    return std::tie(p, n0, n1, n2, esz, kind) < std::tie(o.p, o.n0, o.n1, o.n2, o.esz, o.kind);
  }
};
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_map_cache;

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

bool cached_map(CUtensorMap* out, const MapKey& key, cuuint32_t rank, const void* ptr, const cuuint64_t* dims,
                const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle sw) {
  std::lock_guard<std::mutex> lk(g_map_mu);
  auto it = g_map_cache.find(key);
  if (it != g_map_cache.end()) {
    *out = it->second;
    return true;
  }
  EncodeFn fn = encoder();
  if (!fn) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap m;
  CUresult r = fn(&m, key.esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank,
                  const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  if (g_map_cache.size() > 4096) g_map_cache.clear();
  g_map_cache[key] = m;
  *out = m;
  return true;
}
}  // namespace

bool strided_map(CUtensorMap* out, const void* ptr, const Geom& g, int esz, int axis) {
  if (axis != 0 && axis != 1) return false;
  const int W = 64 / esz;
  const cuuint64_t dims[3] = {(cuuint64_t)g.n[2], (cuuint64_t)g.n[1], (cuuint64_t)g.n[0]};
  const cuuint64_t strides[2] = {(cuuint64_t)g.n[2] * esz, (cuuint64_t)g.n[1] * g.n[2] * esz};
  const cuuint32_t box[3] = {(cuuint32_t)W, (cuuint32_t)(axis == 1 ? g.n[1] : 1),
                             (cuuint32_t)(axis == 0 ? g.n[0] : 1)};
  return cached_map(out, MapKey{reinterpret_cast<uintptr_t>(ptr), g.n[0], g.n[1], g.n[2], esz, axis}, 3, ptr, dims,
                    strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

bool row_map(CUtensorMap* out, const void* ptr, const Geom& g, int esz, int rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)g.n[2], (cuuint64_t)g.n[0] * g.n[1]};
  const cuuint64_t strides[1] = {(cuuint64_t)g.n[2] * esz};
  const cuuint32_t box[2] = {(cuuint32_t)g.n[2], (cuuint32_t)rows};
  return cached_map(out, MapKey{reinterpret_cast<uintptr_t>(ptr), g.n[0], g.n[1], g.n[2], esz, 100 + rows}, 2, ptr,
                    dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

bool prof_active() { return prof().on; }

// Bumped by every change of an autotuner choice: graphs captured before
// hold the old kernels and are rebuilt.
std::atomic<int> g_tune_gen{0};

namespace {
// (cap << 1) | pencil per kernel class and pencil length
std::atomic<int> g_tuned[kcCount][kNumL];
bool tuned_key(int cls, int L) { return cls >= 0 && cls < kcCount && L >= 8 && L <= 256; }
}
int tuned_cap(int cls, int L) { return tuned_key(cls, L) ? (g_tuned[cls][lidx(L)].load() >> 1) : 0; }
bool tuned_pencil(int cls, int L) { return tuned_key(cls, L) && (g_tuned[cls][lidx(L)].load() & 1); }
void set_tuned(int cls, int L, int cap, bool pencil) {
  if (tuned_key(cls, L)) g_tuned[cls][lidx(L)].store(((cap < 0 ? 0 : cap) << 1) | (pencil ? 1 : 0));
  ++g_tune_gen;
}
void clear_tuned() {
  for (int c = 0; c < kcCount; ++c)
    for (int i = 0; i < kNumL; ++i) g_tuned[c][i].store(0);
  ++g_tune_gen;
}

int prof_begin(int cls, cudaStream_t s) {
  Profiler& p = prof();
  if (!p.on) return -1;
  std::lock_guard<std::mutex> lk(p.mu);
  Profiler::Rec r{cls, p.get(), p.get()};
  cudaEventRecord(r.a, s);
  p.pending.push_back(r);
  return (int)p.pending.size() - 1;
}

void prof_end(int token, cudaStream_t s) {
  if (token < 0) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (token < (int)p.pending.size()) cudaEventRecord(p.pending[token].b, s);
}

namespace {

constexpr double kTwoPi = kTwoPiHost;

// Bump allocator over the caller's workspace (256-byte alignment).
struct Carve {
  char* base;
  size_t off = 0, cap;
  bool measure;
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = measure ? nullptr : base + off;
    off += bytes;
    return p;
  }
};


enum Field {
  F_KAPPA1, F_RHO1, F_C0, F_D, F_ALPHA, F_AB, F_WS, F_CN, F_CS,
  F_X, F_R, F_P, F_Q, F_W1, F_W2, F_CH, F_CHS, F_U,
  // state-solve guesses: increments and their (I - sA) images of the last
  // two steps (slot = step parity), and the right-hand side of the solve
  F_GD0, F_GD1, F_GG0, F_GG1, F_FS,
  F_COUNT
};
constexpr int kAnatomyFields = 6;   // m_WM, m_GM, m_CSF, m_D,WM, m_D,GM, m_D,CSF
constexpr int kCouplingFields = 2;  // per-voxel k_f and rho_f integrands of the adjoint

}  // namespace

// Whether the next PCG solve starts from the guess already in x.
__global__ void k_set_keep(PcgState* st, int keep) { st->keep_x = keep; }

// Tiles of the TMA passes on which kappa1 is not identically zero.  The
// operator d_a(kappa d_a u) and the k_f integrand kappa grad(a).grad(w)
// vanish exactly on the others (the brain sits inside the periodic box with
// kappa = 0 outside, Sec. 2.1 and 3.3), so those passes skip them.
//   f0: strided tiles of axis 0, index i1 * nb + i2 / W
//   f1: strided tiles of axis 1, index i0 * nb + i2 / W
//   fr: row tiles of the contiguous axis, index (i0 n1 + i1) / rows
template <typename T>
__global__ void k_kappa_tiles(const T* __restrict__ kappa, Geom g, int W, int rows, int* f0, int* f1, int* fr) {
  const int n1 = g.n[1], n2 = g.n[2];
  const int nb = n2 / W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.nn;
       i += (long long)gridDim.x * blockDim.x) {
    if (kappa[i] == T(0)) continue;
    const int i2 = int(i % n2);
    const long long row = i / n2;
    const int i1 = int(row % n1), i0 = int(row / n1);
    if (nb > 0) {
      f0[i1 * nb + i2 / W] = 1;
      f1[i0 * nb + i2 / W] = 1;
    }
    fr[row / rows] = 1;
  }
}

// Rows per tile of the contiguous-axis TMA kernels for pencil length L.
template <typename T>
int row_tile_rows(int L) {
  switch (L) {
    case 8: return TmaRowShape<T, 8>::ROWS;
    case 16: return TmaRowShape<T, 16>::ROWS;
    case 32: return TmaRowShape<T, 32>::ROWS;
    case 64: return TmaRowShape<T, 64>::ROWS;
    case 96: return TmaRowShape<T, 96>::ROWS;
    case 128: return TmaRowShape<T, 128>::ROWS;
    default: return TmaRowShape<T, 256>::ROWS;
  }
}

struct EngineBase {
  virtual ~EngineBase() {}
  rd_config cfg{};
  int np = 0;
  Geom g{};
  long long nn = 0;
  cudaStream_t stream = nullptr;
  char err[512] = {0};
  int last_iters = 0, last_solves = 0, last_graph_solves = 0;
  bool capturing = false;   // enqueue into a stream capture (batch graph)
  bool have_tissue = false, have_basis = false, have_data = false, have_mdata = false;
  bool have_traj = false, have_grad = false;
  double theta_kf = 0, theta_rho = 0;
  std::vector<double> theta_p, last_grad;
  bool nonconv = false;
  // tiles of the TMA passes where kappa1 is not identically zero (strided
  // axis 0, strided axis 1, contiguous-axis row tiles), and all tiles
  long long active_tiles[3] = {0, 0, 0};
  long long all_tiles[3] = {0, 0, 0};

  virtual rd_status set_tissue(const double*, const double*, const double*) = 0;
  virtual rd_status set_basis(const double*, double) = 0;
  virtual rd_status set_data(const double*) = 0;
  virtual rd_status set_anatomy_data(const double*, const double*, const double*) = 0;
  virtual rd_status set_precond_scale(double) = 0;
  virtual rd_status coupling_field(double*, double*, double*) = 0;
  virtual rd_status forward(const double*, double, double, double*, double*) = 0;
  virtual rd_status adjoint(double*) = 0;
  virtual rd_status hessvec(const double*, double, double, const double*, double*) = 0;
  virtual rd_status apply_operator(double, const double*, double*) = 0;
  virtual rd_status apply_precond(double, const double*, double*) = 0;
  virtual rd_status batch_enqueue(const double*, double, double, cudaStream_t) = 0;
  virtual rd_status batch_finish(double*, double*) = 0;
  virtual void batch_prepare(const double*, double, double) = 0;
  virtual rd_status autotune(int, int*, int*, int) = 0;
  virtual bool warm() const = 0;
};

template <typename T>
struct Engine : EngineBase {
  using L_ = Launch<T>;
  void* ws = nullptr;
  bool own_ws = false;
  Params* prm = nullptr;
  Params* hprm = nullptr;   // pinned host mirror
  PcgState* st = nullptr;
  PcgState* hst = nullptr;  // pinned host mirror
  double* part = nullptr;
  unsigned int* counter = nullptr;
  cpx<T>* twA[kNumL] = {};
  cpx<T>* twB[kNumL] = {};
  double* fac = nullptr;
  T* fac_t = nullptr;   // the same factors in T (per-voxel sums of the basis)
  double* pdev = nullptr;
  double* gp = nullptr;
  double* phit_part = nullptr;
  double* stage[3] = {};
  T* f[F_COUNT] = {};
  T* anat[kAnatomyFields] = {};   // Moving-Atlas fields (cfg.moving_atlas)
  T* qf[kCouplingFields] = {};    // coupling integrands (cfg.coupling)
  bool have_q = false;
  double q_kf = 0.0, q_rho = 0.0;
  double kbar_base = 0.0, kbar_factor = 1.0;   // preconditioner constant and its user scale
  std::vector<T*> slots;   // checkpoint storage
  int nmax = 0;
  double sigma = 0;
  int stride = 0, nseg = 0;   // checkpoint stride and number of stored states
  int seg_loaded = -1;        // segment whose c** are in the segment slots
  // one PCG solve as a CUDA graph: memset + setup, then a device-side WHILE
  // node over the iteration body (built on first use, reused by every solve)
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  int pcg_gen = 0;   // autotuner generation the graph was captured under
  bool warm_next = false;   // the next pcg() starts from the guess in F_X
  bool graph_failed = false;
  int host_solves = 0;
  cudaStream_t cap_stream = nullptr;    // internal stream used only for capture
  cudaStream_t body_stream = nullptr;   // captures WHILE bodies during a batch capture
  double* hp = nullptr;                 // pinned host copy of p (or v)
  double* hgp = nullptr;                // pinned host copy of g_p
  double* hv = nullptr;                 // pinned host copy of a direction v
  // tiles where kappa1 is not identically zero (see k_kappa_tiles): lists of
  // the strided tiles of axes 0 and 1, a flag per row tile, and the two list
  // lengths (device)
  int* tl[2] = {};
  int* rowact = nullptr;
  int* tcount = nullptr;

  // ------------------------------------------------------------ set-up
  static size_t layout(Carve& c, const rd_config& cfg, int np, Engine* e) {
    const long long nn = (long long)cfg.n[0] * cfg.n[1] * cfg.n[2];
    const int nmax = std::max(cfg.n[0], std::max(cfg.n[1], cfg.n[2]));
    auto put = [&](void** dst, size_t bytes) {
      void* p = c.take(bytes);
      if (e) *dst = p;
    };
    void* dummy;
    put(e ? (void**)&e->prm : &dummy, sizeof(Params));
    put(e ? (void**)&e->st : &dummy, sizeof(PcgState));
    put(e ? (void**)&e->part : &dummy, sizeof(double) * kMaxBlocks * 4);
    put(e ? (void**)&e->counter : &dummy, sizeof(unsigned int) * 64);
    for (int i = 0; i < kNumL; ++i) {
      const int L = slot_length(i);
      put(e ? (void**)&e->twA[i] : &dummy, sizeof(cpx<T>) * L);
      put(e ? (void**)&e->twB[i] : &dummy, sizeof(cpx<T>) * L);
    }
    put(e ? (void**)&e->fac : &dummy, sizeof(double) * size_t(np) * 3 * nmax);
    put(e ? (void**)&e->fac_t : &dummy, sizeof(T) * size_t(np) * 3 * nmax);
    put(e ? (void**)&e->pdev : &dummy, sizeof(double) * (np + 2));
    put(e ? (void**)&e->gp : &dummy, sizeof(double) * (np + 2));
    put(e ? (void**)&e->phit_part : &dummy, sizeof(double) * size_t(np) * cfg.n[0]);
    {
      const int W = 64 / int(sizeof(T));
      const long long nb = (cfg.n[2] + W - 1) / W;
      put(e ? (void**)&e->tl[0] : &dummy, sizeof(int) * size_t(cfg.n[1] * nb));
      put(e ? (void**)&e->tl[1] : &dummy, sizeof(int) * size_t(cfg.n[0] * nb));
      put(e ? (void**)&e->rowact : &dummy, sizeof(int) * size_t(cfg.n[0]) * cfg.n[1]);
      put(e ? (void**)&e->tcount : &dummy, sizeof(int) * 4);
    }
    for (int i = 0; i < 3; ++i) put(e ? (void**)&e->stage[i] : &dummy, sizeof(double) * nn);
    for (int i = 0; i < F_COUNT; ++i) put(e ? (void**)&e->f[i] : &dummy, sizeof(T) * nn);
    if (cfg.moving_atlas)
      for (int i = 0; i < kAnatomyFields; ++i) put(e ? (void**)&e->anat[i] : &dummy, sizeof(T) * nn);
    if (cfg.coupling)
      for (int i = 0; i < kCouplingFields; ++i) put(e ? (void**)&e->qf[i] : &dummy, sizeof(T) * nn);
    int nslots;
    if (cfg.ckpt_stride <= 0 || cfg.ckpt_stride >= cfg.nt) {
      nslots = cfg.nt;
    } else {
      const int s = cfg.ckpt_stride;
      nslots = (cfg.nt + s - 1) / s + s;
    }
    for (int i = 0; i < nslots; ++i) {
      void* p = c.take(sizeof(T) * nn);
      if (e) e->slots.push_back(reinterpret_cast<T*>(p));
    }
    return c.off + 256;
  }

  rd_status fail(rd_status s, const char* msg) {
    snprintf(err, sizeof(err), "%s", msg);
    return s;
  }
  rd_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(err, sizeof(err), "%s: %s", where, cudaGetErrorString(e));
    return RD_ERR_CUDA;
  }

  rd_status init(const rd_config& c, int np_, void* workspace, size_t bytes, cudaStream_t s) {
    cfg = c;
    np = np_;
    stream = s;
    for (int a = 0; a < 3; ++a) g.n[a] = cfg.n[a];
    nn = g.nn = (long long)cfg.n[0] * cfg.n[1] * cfg.n[2];
    nmax = std::max(cfg.n[0], std::max(cfg.n[1], cfg.n[2]));
    Carve m{nullptr, 0, 0, true};
    const size_t need = layout(m, cfg, np, nullptr);
    if (!workspace) {
      cudaError_t e = cudaMalloc(&ws, need);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
      own_ws = true;
    } else {
      if (bytes < need) return fail(RD_ERR_NOMEM, "workspace smaller than rd_workspace_size()");
      if (reinterpret_cast<uintptr_t>(workspace) & 255) return fail(RD_ERR_ARG, "workspace not 256-byte aligned");
      ws = workspace;
    }
    Carve cv{reinterpret_cast<char*>(ws), 0, need, false};
    layout(cv, cfg, np, this);
    if (cfg.ckpt_stride > 0 && cfg.ckpt_stride < cfg.nt) {
      stride = cfg.ckpt_stride;
      nseg = (cfg.nt + stride - 1) / stride;
    } else {
      stride = 0;
      nseg = 0;
    }
    cudaError_t e;
    if ((e = cudaMallocHost(&hprm, sizeof(Params))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hst, sizeof(PcgState))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hp, sizeof(double) * (np + 2))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hgp, sizeof(double) * (np + 2))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&hv, sizeof(double) * (np + 2))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    memset(hprm, 0, sizeof(Params));
    memset(hst, 0, sizeof(PcgState));
    hprm->s = 0.5 * cfg.t_end / cfg.nt;
    hprm->h3 = kTwoPi * kTwoPi * kTwoPi / double(nn);
    hprm->inv_nn = 1.0 / double(nn);
    hst->rtol2 = cfg.pcg_rtol * cfg.pcg_rtol;
    hst->maxit = cfg.pcg_maxit;
    if ((e = cudaMemcpyAsync(prm, hprm, sizeof(Params), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload params");
    if ((e = cudaMemcpyAsync(st, hst, sizeof(PcgState), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload pcg state");
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 64, stream)) != cudaSuccess)
      return cuda_fail(e, "memset counters");
    // twiddle tables, computed in FP64 on the host
    std::vector<cpx<T>> ta, tb;
    for (int i = 0; i < kNumL; ++i) {
      const int L = slot_length(i);
      build_twiddles<T>(L, ta, tb);
      if ((e = cudaMemcpyAsync(twA[i], ta.data(), sizeof(cpx<T>) * L, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      if ((e = cudaMemcpyAsync(twB[i], tb.data(), sizeof(cpx<T>) * L, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    }
    return RD_OK;
  }

  ~Engine() override {
    if (pcg_exec) cudaGraphExecDestroy(pcg_exec);
    if (pcg_graph) cudaGraphDestroy(pcg_graph);
    if (hprm) cudaFreeHost(hprm);
    if (hst) cudaFreeHost(hst);
    if (hp) cudaFreeHost(hp);
    if (hgp) cudaFreeHost(hgp);
    if (hv) cudaFreeHost(hv);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (body_stream) cudaStreamDestroy(body_stream);
    if (own_ws && ws) cudaFree(ws);
  }

  // ------------------------------------------------------------ helpers
  Fin fin(int kind, int slot = 0, double scale = 1.0, double* target = nullptr) {
    Fin r;
    r.kind = kind;
    r.slot = slot;
    r.scale = scale;
    r.st = st;
    r.prm = prm;
    r.part = part;
    r.counter = counter;
    r.target = target;
    return r;
  }

  // copy an FP64 field (host or device) into staging slot i; returns the
  // device pointer to read from
  cudaError_t stage_in(const double* src, int i, const double** dev) {
    if (is_device_ptr(src)) {
      *dev = src;
      return cudaSuccess;
    }
    *dev = stage[i];
    return cudaMemcpyAsync(stage[i], src, sizeof(double) * nn, cudaMemcpyHostToDevice, stream);
  }

  cudaError_t field_out(const T* src, double* dst, double scale) {
    cudaError_t e;
    if (is_device_ptr(dst)) return L_::to_f64(src, dst, nn, scale, stream);
    if ((e = L_::to_f64(src, stage[0], nn, scale, stream)) != cudaSuccess) return e;
    return cudaMemcpyAsync(dst, stage[0], sizeof(double) * nn, cudaMemcpyDeviceToHost, stream);
  }

  cudaError_t upload_params() {
    return cudaMemcpyAsync(prm, hprm, sizeof(Params), cudaMemcpyHostToDevice, stream);
  }

  // out = c0 * (use_kf ? k_f : 1) * s * A1 u, A1 = div(kappa1 grad .)
  cudaError_t apply3(const T* u, T* out, double c0, int use_kf) {
    for (int axis : {2, 1, 0}) {
      OpArgs<T> a{};
      a.u = u;
      a.kappa = f[F_KAPPA1];
      a.acc_in = (axis == 2) ? nullptr : out;
      a.out = out;
      a.c0 = c0;
      a.use_kf = use_kf;
      a.a_self = 0;
      a.reduce = 0;
      a.axis = axis;
      a.g = g;
      const int L = g.n[axis];
      a.twA = twA[lidx(L)];
      a.twB = twB[lidx(L)];
      a.prm = prm;
      a.fin = fin(kFinNone);
      if (axis != 2) {
        a.tiles = tl[axis];
        a.ntiles_act = &tcount[axis];
      }
      cudaError_t e = L_::op(L, a, stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  DhtArgs<T> dht_args(int axis, const T* in, T* out) {
    DhtArgs<T> a{};
    a.in = in;
    a.out = out;
    a.axis = axis;
    a.g = g;
    const int L = g.n[axis];
    a.twA = twA[lidx(L)];
    a.twB = twB[lidx(L)];
    a.prm = prm;
    a.st = st;
    return a;
  }

  // ---- PCG kernels (shared by the host-driven loop and the graph) ------
  cudaError_t enqueue_setup(unsigned long long cond) {
    cudaError_t e;
    // x = 0 unless the solve starts from a guess (st->keep_x, set by pcg())
    if ((e = L_::x_init(f[F_X], st, nn, stream)) != cudaSuccess) return e;
    DhtArgs<T> a = dht_args(2, f[F_R], f[F_W1]);
    a.fin = fin(kFinSetup);
    a.fin.cond = cond;
    return L_::dht(g.n[2], kDhtSetup, a, stream);
  }

  cudaError_t enqueue_iteration(unsigned long long cond) {
    cudaError_t e;
    T *X = f[F_X], *R = f[F_R], *P = f[F_P], *Q = f[F_Q], *W1 = f[F_W1], *W2 = f[F_W2];
    {
      DhtArgs<T> a = dht_args(1, W1, W2);
      if ((e = L_::dht(g.n[1], kDhtPlain, a, stream)) != cudaSuccess) return e;
    }
    {
      DhtArgs<T> a = dht_args(0, W2, W1);
      a.fin = fin(kFinRz);
      if ((e = L_::dht(g.n[0], kDhtSym, a, stream)) != cudaSuccess) return e;
    }
    {
      DhtArgs<T> a = dht_args(1, W1, W2);
      if ((e = L_::dht(g.n[1], kDhtPlain, a, stream)) != cudaSuccess) return e;
    }
    {
      PcgOpxArgs<T> a{};
      a.w = W2;
      a.p = P;
      a.q = Q;
      a.x = X;   // the previous iteration's x += alpha p rides on this kernel
      a.kappa = f[F_KAPPA1];
      a.g = g;
      a.twA = twA[lidx(g.n[2])];
      a.twB = twB[lidx(g.n[2])];
      a.prm = prm;
      a.st = st;
      a.fin = fin(kFinPqAdd, 0, 1.0 / (double(g.n[2]) * g.n[2]));
      a.rowact = rowact;
      if ((e = L_::pcg_opx(g.n[2], a, stream)) != cudaSuccess) return e;
    }
    for (int axis : {1, 0}) {
      OpArgs<T> a{};
      a.u = P;
      a.kappa = f[F_KAPPA1];
      a.acc_in = Q;
      a.out = Q;
      a.c0 = -1.0;
      a.use_kf = 1;
      a.a_self = 0;
      a.reduce = 1;
      a.axis = axis;
      a.g = g;
      a.twA = twA[lidx(g.n[axis])];
      a.twB = twB[lidx(g.n[axis])];
      a.prm = prm;
      a.fin = fin(axis == 0 ? kFinPqLast : kFinPqAdd, 0, 1.0 / (double(g.n[axis]) * g.n[axis]));
      a.tiles = tl[axis];
      a.ntiles_act = &tcount[axis];
      if ((e = L_::op(g.n[axis], a, stream)) != cudaSuccess) return e;
    }
    {
      DhtArgs<T> a = dht_args(2, nullptr, W1);
      a.r = R;
      a.q = Q;
      a.fin = fin(kFinRr);
      a.fin.cond = cond;
      if ((e = L_::dht(g.n[2], kDhtUpdate, a, stream)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // Capture setup + WHILE(iteration) into one executable graph.
  bool build_pcg_graph() {
    // capture on an internal stream (the caller's stream may be the legacy
    // default stream, which cannot be captured); the graph is launched on
    // the caller's stream
    cudaStream_t user = stream;
    stream = cap_stream;
    bool ok = build_pcg_graph_on_stream();
    stream = user;
    return ok;
  }

  bool build_pcg_graph_on_stream() {
    cudaGraph_t gph = nullptr, body = nullptr, cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t cond_node = nullptr, leaf = nullptr;
    size_t nnodes = 0;
    std::vector<cudaGraphNode_t> nodes;
    bool ok = false;
    do {
      if (cudaGraphCreate(&gph, 0) != cudaSuccess) break;
      if (cudaGraphConditionalHandleCreate(&h, gph, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
      if (cudaStreamBeginCaptureToGraph(stream, gph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        break;
      cudaError_t e1 = enqueue_setup(h);
      cudaError_t e2 = cudaStreamEndCapture(stream, &cap);
      if (e1 != cudaSuccess || e2 != cudaSuccess) break;
      if (cudaGraphGetNodes(gph, nullptr, &nnodes) != cudaSuccess || nnodes == 0) break;
      nodes.resize(nnodes);
      if (cudaGraphGetNodes(gph, nodes.data(), &nnodes) != cudaSuccess) break;
      for (auto nd : nodes) {
        size_t nd_out = 0;
        if (cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out) == cudaSuccess && nd_out == 0) leaf = nd;
      }
      if (!leaf) break;
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if (cudaGraphAddNode(&cond_node, gph, &leaf, nullptr, 1, &cp) != cudaSuccess) break;
      body = cp.conditional.phGraph_out[0];
      if (cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        break;
      e1 = enqueue_iteration(h);
      e2 = cudaStreamEndCapture(stream, &cap);
      if (e1 != cudaSuccess || e2 != cudaSuccess) break;
      if (cudaGraphInstantiate(&exec, gph, 0) != cudaSuccess) break;
      ok = true;
    } while (false);
    if (!ok) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(stream, &junk);
        if (junk && junk != gph) cudaGraphDestroy(junk);
      }
      cudaGetLastError();
      if (gph) cudaGraphDestroy(gph);
      return false;
    }
    pcg_graph = gph;
    pcg_exec = exec;
    return true;
  }

  // Inside a stream capture: setup on the capturing stream, then a WHILE
  // node whose body (captured on body_stream) is one PCG iteration.
  rd_status pcg_captured() {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e;
    if ((e = cudaStreamGetCaptureInfo(stream, &cs, nullptr, &cg, &deps, nullptr, &nd)) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
      return cuda_fail(e == cudaSuccess ? cudaErrorStreamCaptureInvalidated : e, "capture info");
    cudaGraphConditionalHandle h = 0;
    if ((e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
      return cuda_fail(e, "conditional handle");
    if ((e = enqueue_setup(h)) != cudaSuccess) return cuda_fail(e, "pcg setup");
    if ((e = cudaStreamGetCaptureInfo(stream, &cs, nullptr, &cg, &deps, nullptr, &nd)) != cudaSuccess)
      return cuda_fail(e, "capture info");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn = nullptr;
    if ((e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp)) != cudaSuccess) return cuda_fail(e, "while node");
    if ((e = cudaStreamUpdateCaptureDependencies(stream, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      return cuda_fail(e, "capture dependencies");
    cudaGraph_t body = cp.conditional.phGraph_out[0], junk = nullptr;
    cudaStream_t outer = stream;
    stream = body_stream;
    e = cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    cudaError_t e2 = (e == cudaSuccess) ? enqueue_iteration(h) : e;
    cudaError_t e3 = cudaStreamEndCapture(stream, &junk);
    stream = outer;
    if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
      return cuda_fail(e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3), "while body");
    if ((e = enqueue_final()) != cudaSuccess) return cuda_fail(e, "pcg final update");
    ++last_graph_solves;
    return RD_OK;
  }

  // The last deferred x += alpha p of a solve (see DhtArgs).
  cudaError_t enqueue_final() { return L_::cg_final(f[F_X], f[F_P], st, nn, stream); }

  // Preconditioned CG on (I - s k_f A1) x = f with x0 = 0; f in F_R on entry;
  // the solution is left in F_X and the final residual in F_R.  After two
  // host-driven solves (which also warm every launcher's caches) the solve
  // runs as one graph launch with the iteration loop on the device.
  rd_status pcg() {
    cudaError_t e;
    ++last_solves;
    k_set_keep<<<1, 1, 0, stream>>>(st, warm_next ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pcg start");
    if (capturing) return pcg_captured();
    const bool profiling = prof_active();
    if (!profiling && !graph_failed && host_solves >= 2) {
      if (pcg_exec && pcg_gen != g_tune_gen.load()) {
        cudaGraphExecDestroy(pcg_exec);
        cudaGraphDestroy(pcg_graph);
        pcg_exec = nullptr;
        pcg_graph = nullptr;
      }
      if (!pcg_exec) {
        pcg_gen = g_tune_gen.load();
        if (!build_pcg_graph()) graph_failed = true;
      }
      if (pcg_exec) {
        if ((e = cudaGraphLaunch(pcg_exec, stream)) != cudaSuccess) return cuda_fail(e, "pcg graph launch");
        if ((e = enqueue_final()) != cudaSuccess) return cuda_fail(e, "pcg final update");
        ++last_graph_solves;
        return RD_OK;
      }
    }
    ++host_solves;
    if ((e = enqueue_setup(0)) != cudaSuccess) return cuda_fail(e, "pcg setup");
    for (int guard = 0;; ++guard) {
      if (guard > cfg.pcg_maxit + 2) return fail(RD_ERR_CUDA, "PCG state did not advance");
      if ((e = cudaMemcpyAsync(hst, st, sizeof(PcgState), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read pcg state");
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "pcg sync");
      if (hst->sticky == kStTimeout) return fail(RD_ERR_CUDA, "a TMA wait timed out");
      if (hst->done) break;
      if ((e = enqueue_iteration(0)) != cudaSuccess) return cuda_fail(e, "pcg iteration");
    }
    if ((e = enqueue_final()) != cudaSuccess) return cuda_fail(e, "pcg final update");
    return RD_OK;
  }

  PwArgs<T> pw_args() {
    PwArgs<T> a{};
    a.rho1 = f[F_RHO1];
    a.nn = nn;
    a.prm = prm;
    if (have_mdata)
      for (int j = 0; j < 3; ++j) {
        a.m[j] = anat[j];
        a.md[j] = anat[3 + j];
      }
    return a;
  }

  // storage of c** for step n and the "previous" pointer of step n
  T* css_slot(int n) { return stride ? slots[nseg + (n % stride)] : slots[n]; }
  void prev_of(int n, const T** prev, int* is_state) {
    if (n == 0) {
      *prev = stride ? slots[0] : f[F_C0];
      *is_state = 1;
    } else if (stride && n % stride == 0) {
      *prev = slots[n / stride];
      *is_state = 1;
    } else {
      *prev = css_slot(n - 1);
      *is_state = 0;
    }
  }

  // st->bb = ||x + cy y||^2: the Crank-Nicolson right-hand side of the next
  // solve (forward: b = c* + f / 2 with f = 2 s A c*; adjoint: b = alpha**)
  cudaError_t rhs_norm(const T* x, const T* y, double cy) {
    NormArgs<T> a{};
    a.x = x;
    a.y = y;
    a.cy = cy;
    a.nn = nn;
    a.fin = fin(kFinSet, 0, 1.0, &st->bb);
    return L_::normsq(a, stream);
  }

  // Order of the initial guess of step n's state solve: the steps since the
  // last restart (step 0, multiples of guess_restart, checkpoint segment
  // starts), at most 2; -1 when guesses are off.
  int guess_order(int n) const {
    if (cfg.guess_restart < 0) return -1;
    int n0 = 0;
    if (cfg.guess_restart > 0) n0 = std::max(n0, n - n % cfg.guess_restart);
    if (stride) n0 = std::max(n0, n - n % stride);
    return std::min(n - n0, 2);
  }

  rd_status fwd_step(int n) {
    cudaError_t e;
    rd_status rs;
    const T* prev;
    int is_state;
    prev_of(n, &prev, &is_state);
    PwArgs<T> a = pw_args();
    a.prev = prev;
    a.prev_is_state = is_state;
    a.out0 = f[F_CS];
    if ((e = L_::pw(kPwFwdPre, a, stream)) != cudaSuccess) return cuda_fail(e, "fwd pre");
    if ((e = apply3(f[F_CS], f[F_R], 2.0, 1)) != cudaSuccess) return cuda_fail(e, "fwd rhs");
    if ((e = rhs_norm(f[F_CS], f[F_R], 0.5)) != cudaSuccess) return cuda_fail(e, "fwd rhs norm");
    const int order = guess_order(n);
    const int s1 = (n + 1) & 1, s0 = n & 1;   // slots of steps n - 1 and n - 2 (and n)
    if (order >= 0 && (e = L_::guess(f[F_R], f[F_X], f[F_FS], f[F_GD0 + s1], f[F_GD0 + s0], f[F_GG0 + s1],
                                     f[F_GG0 + s0], order, nn, stream)) != cudaSuccess)
      return cuda_fail(e, "guess");
    warm_next = order >= 0;
    rs = pcg();
    warm_next = false;
    if (rs != RD_OK) return rs;
    if (order >= 0 &&
        (e = L_::guess_keep(f[F_GD0 + s0], f[F_GG0 + s0], f[F_X], f[F_R], f[F_FS], nn, stream)) != cudaSuccess)
      return cuda_fail(e, "keep guess");
    PwArgs<T> b = pw_args();
    b.a = f[F_CS];
    b.b = f[F_X];
    b.out0 = css_slot(n);
    if ((e = L_::pw(kPwFwdPost, b, stream)) != cudaSuccess) return cuda_fail(e, "fwd post");
    return RD_OK;
  }

  // store the state c_n of a segment start (checkpoint mode)
  rd_status store_state(int n) {
    const T* prev;
    int is_state;
    if (n == 0) return RD_OK;   // slot 0 written from Phi p
    prev = css_slot(n - 1);
    is_state = 0;
    PwArgs<T> a = pw_args();
    a.prev = prev;
    a.prev_is_state = is_state;
    a.out0 = slots[n / stride];
    cudaError_t e = L_::pw(kPwState, a, stream);
    return e == cudaSuccess ? RD_OK : cuda_fail(e, "store state");
  }

  rd_status run_segment(int k) {   // recompute c** of segment k into the segment slots
    rd_status rs;
    const int n0 = k * stride, n1 = std::min(cfg.nt, n0 + stride);
    for (int n = n0; n < n1; ++n)
      if ((rs = fwd_step(n)) != RD_OK) return rs;
    seg_loaded = k;
    return RD_OK;
  }

  rd_status run_forward(const double* p, double k_f, double rho_f) {
    have_q = false;
    cudaError_t e;
    rd_status rs;
    if (!have_tissue || !have_basis) return fail(RD_ERR_STATE, "rd_set_tissue and rd_set_basis are required");
    hprm->k_f = k_f;
    hprm->rho_f = rho_f;
    hprm->v_k = hprm->v_rho = 0.0;
    for (double& x : hprm->acc) x = 0.0;
    if (p != hp) memcpy(hp, p, sizeof(double) * np);
    if ((e = upload_params()) != cudaSuccess) return cuda_fail(e, "upload params");
    if ((e = cudaMemcpyAsync(pdev, hp, sizeof(double) * np, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload p");
    PhiArgs<T> pa{};
    pa.fac = fac;
    pa.fac_t = fac_t;
    pa.p = pdev;
    pa.out = stride ? slots[0] : f[F_C0];
    pa.np = np;
    pa.nmax = nmax;
    pa.g = g;
    pa.cut = 1e-30;
    if ((e = L_::phi(pa, stream)) != cudaSuccess) return cuda_fail(e, "phi");
    for (int n = 0; n < cfg.nt; ++n) {
      if (stride && n % stride == 0 && (rs = store_state(n)) != RD_OK) return rs;
      if ((rs = fwd_step(n)) != RD_OK) return rs;
    }
    seg_loaded = stride ? (cfg.nt - 1) / stride : -1;
    theta_p.assign(hp, hp + np);
    theta_kf = k_f;
    theta_rho = rho_f;
    have_traj = true;
    have_grad = false;
    return RD_OK;
  }

  // misfit kernel: alpha(1) = d - c(1), acc[misfit], c(1) into F_CS
  rd_status enqueue_misfit() {
    cudaError_t e;
    PwArgs<T> a = pw_args();
    a.a = css_slot(cfg.nt - 1);
    a.d = f[F_D];
    a.out0 = f[F_ALPHA];
    a.out1 = f[F_CS];
    a.reduce = 1;
    a.fin = fin(kFinAcc, kAccMisfit, 0.5 * hprm->h3);
    if ((e = L_::pw(kPwMisfit, a, stream)) != cudaSuccess) return cuda_fail(e, "misfit");
    return RD_OK;
  }

  // misfit, alpha(1) = d - c(1), optional c(1) output
  rd_status finish_forward(double* c1_out, double* misfit) {
    cudaError_t e;
    PwArgs<T> a = pw_args();
    a.a = css_slot(cfg.nt - 1);
    a.d = f[F_D];
    a.out0 = f[F_ALPHA];
    a.out1 = f[F_CS];   // c(1)
    a.reduce = 1;
    a.fin = fin(kFinAcc, kAccMisfit, 0.5 * hprm->h3);
    if ((e = L_::pw(kPwMisfit, a, stream)) != cudaSuccess) return cuda_fail(e, "misfit");
    if (c1_out && (e = field_out(f[F_CS], c1_out, 1.0)) != cudaSuccess) return cuda_fail(e, "c1 out");
    if ((e = cudaMemcpyAsync(hprm, prm, sizeof(Params), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return cuda_fail(e, "read params");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    if (misfit) {
      double reg = 0.0;
      for (double x : theta_p) reg += x * x;
      *misfit = hprm->acc[kAccMisfit] + 0.5 * cfg.beta_p * reg;
    }
    return RD_OK;
  }

  rd_status adj_step(int n, bool acc_q) {
    cudaError_t e;
    rd_status rs;
    const T* prev;
    int is_state;
    prev_of(n, &prev, &is_state);
    const double gscale = -hprm->h3 * hprm->s;
    PwArgs<T> a = pw_args();
    a.a = f[F_ALPHA];
    a.b = css_slot(n);
    a.prev = prev;
    a.prev_is_state = is_state;
    a.out0 = f[F_AB];
    a.out1 = f[F_WS];
    a.out2 = f[F_CN];
    a.q = acc_q ? qf[1] : nullptr;
    a.reduce = 1;
    a.fin = fin(kFinAcc, kAccGrho, gscale);
    if ((e = L_::pw(kPwAdjPre, a, stream)) != cudaSuccess) return cuda_fail(e, "adj pre");
    if ((e = apply3(f[F_AB], f[F_R], 1.0, 1)) != cudaSuccess) return cuda_fail(e, "adj rhs");
    if ((e = rhs_norm(f[F_AB], nullptr, 0.0)) != cudaSuccess) return cuda_fail(e, "adj rhs norm");
    if ((rs = pcg()) != RD_OK) return rs;
    for (int axis : {2, 1, 0}) {
      GradArgs<T> ga{};
      ga.u0 = f[F_AB];
      ga.u1 = f[F_X];
      ga.w = f[F_WS];
      ga.kappa = f[F_KAPPA1];
      ga.q = acc_q ? qf[0] : nullptr;
      ga.qscale = hprm->s;
      ga.axis = axis;
      ga.g = g;
      ga.twA = twA[lidx(g.n[axis])];
      ga.twB = twB[lidx(g.n[axis])];
      ga.fin = fin(kFinAcc, kAccGk, hprm->s * hprm->h3);
      if (axis != 2) {
        ga.tiles = tl[axis];
        ga.ntiles_act = &tcount[axis];
      }
      if ((e = L_::grad(g.n[axis], ga, stream)) != cudaSuccess) return cuda_fail(e, "grad pass");
    }
    PwArgs<T> b = pw_args();
    b.a = f[F_AB];
    b.b = f[F_X];
    b.d = f[F_R];
    b.prev = f[F_CN];
    b.prev_is_state = 1;
    b.out0 = f[F_ALPHA];
    b.q = acc_q ? qf[1] : nullptr;
    b.reduce = 1;
    b.fin = fin(kFinAcc, kAccGrho, gscale);
    if ((e = L_::pw(kPwAdjPost, b, stream)) != cudaSuccess) return cuda_fail(e, "adj post");
    return RD_OK;
  }

  // reverse sweep from alpha(1) in F_ALPHA; g_kf, g_rho into acc, g_p into
  // gp; with acc_q also the per-voxel integrands into the coupling fields
  rd_status run_adjoint(bool acc_q = false) {
    cudaError_t e;
    rd_status rs;
    hprm->acc[kAccGk] = hprm->acc[kAccGrho] = 0.0;
    // zero the two gradient accumulators on the device without touching the rest
    if ((e = cudaMemsetAsync(&prm->acc[kAccGk], 0, 2 * sizeof(double), stream)) != cudaSuccess)
      return cuda_fail(e, "zero acc");
    acc_q = acc_q && cfg.coupling;
    if (acc_q) {
      have_q = false;
      for (int i = 0; i < kCouplingFields; ++i)
        if ((e = cudaMemsetAsync(qf[i], 0, sizeof(T) * nn, stream)) != cudaSuccess) return cuda_fail(e, "zero q");
    }
    if (!stride) {
      for (int n = cfg.nt - 1; n >= 0; --n)
        if ((rs = adj_step(n, acc_q)) != RD_OK) return rs;
    } else {
      for (int k = nseg - 1; k >= 0; --k) {
        if (seg_loaded != k) {
          // the recompute overwrites F_ALPHA's neighbours only; keep alpha
          if ((rs = run_segment(k)) != RD_OK) return rs;
        }
        const int n0 = k * stride, n1 = std::min(cfg.nt, n0 + stride);
        for (int n = n1 - 1; n >= n0; --n)
          if ((rs = adj_step(n, acc_q)) != RD_OK) return rs;
      }
      seg_loaded = -1;
    }
    PhiArgs<T> pa{};
    pa.fac = fac;
    pa.fac_t = fac_t;
    pa.u = f[F_ALPHA];
    pa.part = phit_part;
    pa.np = np;
    pa.nmax = nmax;
    pa.g = g;
    pa.cut = 1e-30;
    if ((e = L_::phit(pa, gp, -hprm->h3, stream)) != cudaSuccess) return cuda_fail(e, "phi^T");
    return RD_OK;
  }

  cudaError_t enqueue_results() {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hgp, gp, sizeof(double) * np, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hprm, prm, sizeof(Params), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
    return cudaMemcpyAsync(hst, st, sizeof(PcgState), cudaMemcpyDeviceToHost, stream);
  }

  void read_results(double* out, const double* vp) {
    for (int i = 0; i < np; ++i) out[i] = hgp[i] + cfg.beta_p * vp[i];
    out[np] = hprm->acc[kAccGk];
    out[np + 1] = hprm->acc[kAccGrho];
  }

  rd_status collect(double* out, const double* vp) {
    cudaError_t e;
    if ((e = enqueue_results()) != cudaSuccess) return cuda_fail(e, "read results");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    read_results(out, vp);
    return RD_OK;
  }

  void begin_call() {
    err[0] = 0;
    last_iters = 0;
    last_solves = 0;
    last_graph_solves = 0;
    nonconv = false;
    // zero the iteration counter and the sticky status (two adjacent ints)
    cudaMemsetAsync(&st->total_it, 0, 2 * sizeof(int), stream);
  }
  rd_status end_call(rd_status s) {
    if (s != RD_OK) return s;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hst, st, sizeof(PcgState), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return cuda_fail(e, "read pcg state");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    last_iters = hst->total_it;
    if (hst->sticky == kStTimeout) return fail(RD_ERR_CUDA, "a TMA wait timed out");
    if (hst->sticky == kStNonFinite) return fail(RD_ERR_NONFINITE, "non-finite value in a PCG solve");
    if (hst->sticky == kStNoConv) {
      snprintf(err, sizeof(err), "a PCG solve reached pcg_maxit");
      return RD_ERR_NOCONV;
    }
    return RD_OK;
  }

  // ------------------------------------------------------------ API
  // Flags of the tiles on which kappa1 is not identically zero, compacted on
  // the host into ascending lists (the order the passes would visit them in).
  cudaError_t kappa_tiles() {
    const int W = 64 / int(sizeof(T));
    const int nb = g.n[2] / W;
    const int rows = row_tile_rows<T>(g.n[2]);
    all_tiles[0] = (long long)g.n[1] * nb;
    all_tiles[1] = (long long)g.n[0] * nb;
    all_tiles[2] = ((long long)g.n[0] * g.n[1] + rows - 1) / rows;
    cudaError_t e;
    for (int a = 0; a < 2; ++a)
      if (all_tiles[a] > 0 && (e = cudaMemsetAsync(tl[a], 0, sizeof(int) * all_tiles[a], stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(rowact, 0, sizeof(int) * all_tiles[2], stream)) != cudaSuccess) return e;
    const int blocks = int(std::min<long long>((nn + 255) / 256, 4096));
    k_kappa_tiles<T><<<blocks, 256, 0, stream>>>(f[F_KAPPA1], g, W, rows, tl[0], tl[1], rowact);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<int> h0(all_tiles[0]), h1(all_tiles[1]);
    if (all_tiles[0] > 0 && (e = cudaMemcpyAsync(h0.data(), tl[0], sizeof(int) * all_tiles[0],
                                                 cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return e;
    if (all_tiles[1] > 0 && (e = cudaMemcpyAsync(h1.data(), tl[1], sizeof(int) * all_tiles[1],
                                                 cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return e;
    std::vector<int> hr(all_tiles[2]);
    if ((e = cudaMemcpyAsync(hr.data(), rowact, sizeof(int) * all_tiles[2], cudaMemcpyDeviceToHost, stream)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
    std::vector<int> l0, l1;
    for (int t = 0; t < (int)h0.size(); ++t)
      if (h0[t]) l0.push_back(t);
    for (int t = 0; t < (int)h1.size(); ++t)
      if (h1[t]) l1.push_back(t);
    long long nr = 0;
    for (int v : hr) nr += v ? 1 : 0;
    active_tiles[0] = (long long)l0.size();
    active_tiles[1] = (long long)l1.size();
    active_tiles[2] = nr;
    int cnt[4] = {int(l0.size()), int(l1.size()), int(nr), 0};
    if (!l0.empty() && (e = cudaMemcpyAsync(tl[0], l0.data(), sizeof(int) * l0.size(), cudaMemcpyHostToDevice,
                                            stream)) != cudaSuccess)
      return e;
    if (!l1.empty() && (e = cudaMemcpyAsync(tl[1], l1.data(), sizeof(int) * l1.size(), cudaMemcpyHostToDevice,
                                            stream)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(tcount, cnt, sizeof(cnt), cudaMemcpyHostToDevice, stream)) != cudaSuccess) return e;
    // the host vectors are pageable and local: wait until the copies are done
    return cudaStreamSynchronize(stream);
  }

  rd_status set_tissue(const double* m0, const double* m1, const double* m2) override {
    cudaError_t e;
    const double* d[3];
    const double* src[3] = {m0, m1, m2};
    for (int i = 0; i < 3; ++i)
      if ((e = stage_in(src[i], i, &d[i])) != cudaSuccess) return cuda_fail(e, "stage tissue");
    CoefArgs<T> a{};
    a.m0 = d[0];
    a.m1 = d[1];
    a.m2 = d[2];
    a.kappa1 = f[F_KAPPA1];
    a.rho1 = f[F_RHO1];
    a.kw0 = cfg.k_w[0];
    a.kw1 = cfg.k_w[1];
    a.kw2 = cfg.k_w[2];
    a.rw0 = cfg.rho_w[0];
    a.rw1 = cfg.rho_w[1];
    a.rw2 = cfg.rho_w[2];
    a.nn = nn;
    a.fin = fin(kFinRatio, 0, 1.0, &prm->kbar1);   // mean of kappa1 where it is positive
    if ((e = L_::coef(a, stream)) != cudaSuccess) return cuda_fail(e, "coefficients");
    if ((e = kappa_tiles()) != cudaSuccess) return cuda_fail(e, "kappa tiles");
    if (cfg.moving_atlas)
      for (int j = 0; j < 3; ++j)
        if ((e = L_::from_f64(d[j], anat[j], nn, stream)) != cudaSuccess) return cuda_fail(e, "tissue maps");
    if ((e = cudaMemcpyAsync(&hprm->kbar1, &prm->kbar1, sizeof(double), cudaMemcpyDeviceToHost, stream)) !=
        cudaSuccess)
      return cuda_fail(e, "read kbar");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    kbar_base = hprm->kbar1;
    have_tissue = true;
    if (kbar_factor != 1.0) {
      rd_status s = set_precond_scale(kbar_factor);
      if (s != RD_OK) return s;
    }
    have_traj = false;
    have_q = false;
    return RD_OK;
  }

  rd_status set_basis(const double* centers, double sig) override {
    if (!(sig > 0)) return fail(RD_ERR_ARG, "sigma must be positive");
    sigma = sig;
    std::vector<double> h(size_t(np) * 3 * nmax, 0.0);
    for (int i = 0; i < np; ++i)
      for (int a = 0; a < 3; ++a)
        for (int x = 0; x < g.n[a]; ++x) {
          double d = kTwoPi * x / g.n[a] - centers[i * 3 + a];
          d -= kTwoPi * std::nearbyint(d / kTwoPi);
          h[(size_t(i) * 3 + a) * nmax + x] = std::exp(-d * d / (2.0 * sig * sig));
        }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(fac, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, stream)) !=
        cudaSuccess)
      return cuda_fail(e, "upload basis");
    std::vector<T> ht(h.begin(), h.end());
    if ((e = cudaMemcpyAsync(fac_t, ht.data(), sizeof(T) * ht.size(), cudaMemcpyHostToDevice, stream)) !=
        cudaSuccess)
      return cuda_fail(e, "upload basis");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    have_basis = true;
    have_traj = false;
    return RD_OK;
  }

  rd_status set_anatomy_data(const double* m0, const double* m1, const double* m2) override {
    if (!cfg.moving_atlas) return fail(RD_ERR_STATE, "rd_set_anatomy_data needs cfg.moving_atlas = 1");
    if (!have_tissue) return fail(RD_ERR_STATE, "rd_set_tissue is required first");
    cudaError_t e;
    const double* src[3] = {m0, m1, m2};
    for (int j = 0; j < 3; ++j) {
      const double* dv;
      if ((e = stage_in(src[j], j, &dv)) != cudaSuccess) return cuda_fail(e, "stage anatomy");
      if ((e = L_::from_f64(dv, anat[3 + j], nn, stream)) != cudaSuccess) return cuda_fail(e, "convert anatomy");
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    have_mdata = true;
    have_q = false;
    return RD_OK;
  }

  // kbar1 = kbar_base * scale, on the host copy (uploaded with the
  // parameters) and on the device (read by the PCG graphs at run time)
  rd_status set_precond_scale(double scale) override {
    kbar_factor = scale;
    if (!have_tissue) return RD_OK;
    hprm->kbar1 = kbar_base * scale;
    cudaError_t e = cudaMemcpyAsync(&prm->kbar1, &hprm->kbar1, sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "preconditioner scale");
    return RD_OK;
  }

  // q_i = k_f k_w,i Q_k + rho_f rho_w,i Q_rho from the integrands of the
  // last gradient adjoint
  rd_status coupling_field(double* q0, double* q1, double* q2) override {
    if (!cfg.coupling) return fail(RD_ERR_STATE, "rd_coupling_field needs cfg.coupling = 1");
    if (!have_q) return fail(RD_ERR_STATE, "rd_coupling_field needs a preceding rd_gradient or rd_adjoint");
    cudaError_t e;
    double* out[3] = {q0, q1, q2};
    for (int j = 0; j < 3; ++j) {
      const double ca = q_kf * cfg.k_w[j], cb = q_rho * cfg.rho_w[j];
      double* dst = is_device_ptr(out[j]) ? out[j] : stage[0];
      if ((e = L_::combine(qf[0], qf[1], ca, cb, dst, nn, stream)) != cudaSuccess) return cuda_fail(e, "combine q");
      if (dst != out[j] &&
          (e = cudaMemcpyAsync(out[j], dst, sizeof(double) * nn, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "q out");
      // the staging buffer is reused by the next class: finish this copy first
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    }
    return RD_OK;
  }

  rd_status set_data(const double* d) override {
    cudaError_t e;
    const double* dv;
    if ((e = stage_in(d, 0, &dv)) != cudaSuccess) return cuda_fail(e, "stage data");
    if ((e = L_::from_f64(dv, f[F_D], nn, stream)) != cudaSuccess) return cuda_fail(e, "convert data");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    have_data = true;
    have_q = false;
    return RD_OK;
  }

  rd_status forward(const double* p, double k_f, double rho_f, double* c1_out, double* misfit) override {
    begin_call();
    rd_status s = run_forward(p, k_f, rho_f);
    if (s != RD_OK) return s;
    if (!have_data) {
      cudaError_t e = cudaMemsetAsync(f[F_D], 0, sizeof(T) * nn, stream);
      if (e != cudaSuccess) return cuda_fail(e, "zero data");
    }
    s = finish_forward(c1_out, have_data ? misfit : nullptr);
    if (s == RD_OK && misfit && !have_data) *misfit = NAN;
    return end_call(s);
  }

  rd_status adjoint(double* alpha0_out) override {
    if (!have_traj) return fail(RD_ERR_STATE, "rd_adjoint needs a preceding rd_forward");
    if (!have_data) return fail(RD_ERR_STATE, "rd_set_data is required");
    const int it0 = last_iters, so0 = last_solves, gs0 = last_graph_solves;
    begin_call();
    rd_status s = run_adjoint(true);
    if (s != RD_OK) return s;
    cudaError_t e;
    if (alpha0_out && (e = field_out(f[F_ALPHA], alpha0_out, 1.0)) != cudaSuccess) return cuda_fail(e, "alpha out");
    last_grad.assign(np + 2, 0.0);
    s = collect(last_grad.data(), theta_p.data());
    if (s == RD_OK) have_grad = true;
    if ((s == RD_OK || s == RD_ERR_NOCONV) && cfg.coupling) {
      have_q = true;
      q_kf = theta_kf;
      q_rho = theta_rho;
    }
    s = end_call(s);
    last_iters += it0;
    last_solves += so0;
    last_graph_solves += gs0;
    return s;
  }

  // ---- autotuner --------------------------------------------------------
  // Times `reps` PCG iterations on this context's buffers for each
  // candidate persistent-grid size (multiples of the SM count) and keeps,
  // per kernel class, the fastest.  The choices apply to every later launch
  // in the process.
  rd_status autotune(int reps, int* caps_out, int* pencil_out, int ncls) override {
    if (!have_tissue) return fail(RD_ERR_STATE, "rd_set_tissue is required");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int kClasses[] = {kcOpStrided, kcPcgOpx, kcDhtPlain, kcDhtSym, kcDhtUpdate};
    // candidates: tile shape (TMA tiles or pencil groups) x persistent grid
    // size (all resident blocks, or 1..8 blocks per SM)
    std::vector<std::pair<int, bool>> cands;
    for (int v = 0; v < 2; ++v) {
      cands.push_back({0, v == 1});
      for (int m = 1; m <= 8; ++m) cands.push_back({m * sms, v == 1});
    }
    double best[kcCount];
    std::pair<int, bool> choice[kcCount];
    for (int c = 0; c < kcCount; ++c) {
      best[c] = 1e300;
      choice[c] = {tuned_cap(c, g.n[2]), tuned_pencil(c, g.n[2])};
    }
    auto set_all = [&](int c, std::pair<int, bool> v) {
      for (int a = 0; a < 3; ++a) set_tuned(c, g.n[a], v.first, v.second);
    };
    cudaError_t e;
    hprm->k_f = (hprm->k_f > 0.0) ? hprm->k_f : 0.05;
    if ((e = upload_params()) != cudaSuccess) return cuda_fail(e, "upload params");
    for (const auto& cand : cands) {
      for (int c : kClasses) set_all(c, cand);
      // a smooth right-hand side: f = A kappa1
      if ((e = apply3(f[F_KAPPA1], f[F_R], 1.0, 1)) != cudaSuccess) return cuda_fail(e, "tune rhs");
      k_set_keep<<<1, 1, 0, stream>>>(st, 0);
      if ((e = enqueue_setup(0)) != cudaSuccess) return cuda_fail(e, "tune setup");
      if ((e = enqueue_iteration(0)) != cudaSuccess) return cuda_fail(e, "tune warm");
      rd_profile_enable(1);
      for (int r = 0; r < reps; ++r)
        if ((e = enqueue_iteration(0)) != cudaSuccess) {
          rd_profile_enable(0);
          return cuda_fail(e, "tune iteration");
        }
      double ms[kcCount];
      long long cnt[kcCount];
      rd_profile_read(ms, cnt, kcCount);
      rd_profile_enable(0);
      for (int c : kClasses)
        if (cnt[c] > 0 && ms[c] / cnt[c] < best[c]) {
          best[c] = ms[c] / cnt[c];
          choice[c] = cand;
        }
    }
    for (int c : kClasses) set_all(c, choice[c]);
    for (int c = 0; c < ncls; ++c) {
      if (caps_out) caps_out[c] = tuned_cap(c, g.n[2]);
      if (pencil_out) pencil_out[c] = tuned_pencil(c, g.n[2]) ? 1 : 0;
    }
    // leave the PCG state clean for the next solve
    if ((e = cudaMemsetAsync(&st->total_it, 0, 2 * sizeof(int), stream)) != cudaSuccess) return cuda_fail(e, "reset");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    return RD_OK;
  }

  // ---- batched gradient -------------------------------------------------
  bool warm() const override { return host_solves >= 2; }

  // Enqueue one whole gradient on `s` (which is being captured into the
  // batch graph): parameters from pinned host memory, forward, misfit,
  // adjoint, Phi^T, and the results back to pinned host memory.
  rd_status batch_enqueue(const double* p, double k_f, double rho_f, cudaStream_t s) override {
    cudaStream_t user = stream;
    stream = s;
    capturing = true;
    begin_call();
    rd_status rs = run_forward(p, k_f, rho_f);
    if (rs == RD_OK) rs = enqueue_misfit();
    if (rs == RD_OK) rs = run_adjoint(true);
    if (rs == RD_OK) {
      cudaError_t e = enqueue_results();
      if (e != cudaSuccess) rs = cuda_fail(e, "results");
    }
    capturing = false;
    stream = user;
    return rs;
  }

  // After the batch graph has run: the same values rd_gradient returns.
  rd_status batch_finish(double* misfit, double* grad) override {
    double reg = 0.0;
    for (int i = 0; i < np; ++i) reg += hp[i] * hp[i];
    if (misfit) *misfit = hprm->acc[kAccMisfit] + 0.5 * cfg.beta_p * reg;
    read_results(grad, hp);
    last_iters = hst->total_it;
    theta_p.assign(hp, hp + np);
    have_traj = true;
    last_grad.assign(grad, grad + np + 2);
    have_grad = true;
    if (cfg.coupling) {
      have_q = true;
      q_kf = hprm_theta_kf;
      q_rho = hprm_theta_rho;
    }
    if (hst->sticky == kStTimeout) return fail(RD_ERR_CUDA, "a TMA wait timed out");
    if (hst->sticky == kStNonFinite) return fail(RD_ERR_NONFINITE, "non-finite value in a PCG solve");
    if (hst->sticky == kStNoConv) return fail(RD_ERR_NOCONV, "a PCG solve reached pcg_maxit");
    return RD_OK;
  }

  // Rewrite the pinned inputs that the batch graph's copy nodes read.
  void batch_prepare(const double* p, double k_f, double rho_f) override {
    hprm->k_f = k_f;
    hprm->rho_f = rho_f;
    hprm->v_k = hprm->v_rho = 0.0;
    for (double& x : hprm->acc) x = 0.0;
    memcpy(hp, p, sizeof(double) * np);
    hprm_theta_kf = k_f;
    hprm_theta_rho = rho_f;
  }
  double hprm_theta_kf = 0, hprm_theta_rho = 0;

  rd_status apply_operator(double k_f, const double* u, double* out) override {
    if (!have_tissue) return fail(RD_ERR_STATE, "rd_set_tissue is required");
    begin_call();
    cudaError_t e;
    hprm->k_f = k_f;
    if ((e = upload_params()) != cudaSuccess) return cuda_fail(e, "upload params");
    const double* dv;
    if ((e = stage_in(u, 1, &dv)) != cudaSuccess) return cuda_fail(e, "stage");
    if ((e = L_::from_f64(dv, f[F_CS], nn, stream)) != cudaSuccess) return cuda_fail(e, "convert");
    if ((e = apply3(f[F_CS], f[F_R], 1.0 / hprm->s, 1)) != cudaSuccess) return cuda_fail(e, "apply");
    if ((e = field_out(f[F_R], out, 1.0)) != cudaSuccess) return cuda_fail(e, "out");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    return RD_OK;
  }

  rd_status apply_precond(double k_f, const double* r, double* out) override {
    if (!have_tissue) return fail(RD_ERR_STATE, "rd_set_tissue is required");
    begin_call();
    cudaError_t e;
    hprm->k_f = k_f;
    if ((e = upload_params()) != cudaSuccess) return cuda_fail(e, "upload params");
    const double* dv;
    if ((e = stage_in(r, 1, &dv)) != cudaSuccess) return cuda_fail(e, "stage");
    if ((e = L_::from_f64(dv, f[F_R], nn, stream)) != cudaSuccess) return cuda_fail(e, "convert");
    DhtArgs<T> a = dht_args(2, f[F_R], f[F_W1]);
    a.fin = fin(kFinSetup);
    if ((e = L_::dht(g.n[2], kDhtSetup, a, stream)) != cudaSuccess) return cuda_fail(e, "dht x");
    a = dht_args(1, f[F_W1], f[F_W2]);
    if ((e = L_::dht(g.n[1], kDhtPlain, a, stream)) != cudaSuccess) return cuda_fail(e, "dht y");
    a = dht_args(0, f[F_W2], f[F_W1]);
    a.fin = fin(kFinRz);
    if ((e = L_::dht(g.n[0], kDhtSym, a, stream)) != cudaSuccess) return cuda_fail(e, "dht z");
    a = dht_args(1, f[F_W1], f[F_W2]);
    if ((e = L_::dht(g.n[1], kDhtPlain, a, stream)) != cudaSuccess) return cuda_fail(e, "dht y");
    a = dht_args(2, f[F_W2], f[F_W1]);
    if ((e = L_::dht(g.n[2], kDhtPlain, a, stream)) != cudaSuccess) return cuda_fail(e, "dht x");
    if ((e = field_out(f[F_W1], out, 1.0)) != cudaSuccess) return cuda_fail(e, "out");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    return RD_OK;
  }

  rd_status hessvec(const double* p, double k_f, double rho_f, const double* v, double* Hv) override {
    begin_call();
    rd_status s;
    cudaError_t e;
    bool same = have_traj && k_f == theta_kf && rho_f == theta_rho && (int)theta_p.size() == np;
    for (int i = 0; same && i < np; ++i) same = (theta_p[i] == p[i]);
    if (!same && (s = run_forward(p, k_f, rho_f)) != RD_OK) return s;
    hprm->k_f = k_f;
    hprm->rho_f = rho_f;
    hprm->v_k = v[np];
    hprm->v_rho = v[np + 1];
    for (double& x : hprm->acc) x = 0.0;
    if ((e = upload_params()) != cudaSuccess) return cuda_fail(e, "upload params");
    memcpy(hv, v, sizeof(double) * np);
    if ((e = cudaMemcpyAsync(pdev, hv, sizeof(double) * np, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload v");
    PhiArgs<T> pa{};
    pa.fac = fac;
    pa.fac_t = fac_t;
    pa.p = pdev;
    pa.out = f[F_CH];
    pa.np = np;
    pa.nmax = nmax;
    pa.g = g;
    pa.cut = 1e-30;
    if ((e = L_::phi(pa, stream)) != cudaSuccess) return cuda_fail(e, "phi v");
    for (int n = 0; n < cfg.nt; ++n) {
      if (stride && n % stride == 0 && seg_loaded != n / stride) {
        if ((s = run_segment(n / stride)) != RD_OK) return s;
      }
      const T* prev;
      int is_state;
      prev_of(n, &prev, &is_state);
      PwArgs<T> a = pw_args();
      a.a = f[F_CH];
      a.b = css_slot(n);
      a.prev = prev;
      a.prev_is_state = is_state;
      a.out0 = f[F_CHS];
      a.out1 = f[F_U];
      if ((e = L_::pw(kPwTlPre, a, stream)) != cudaSuccess) return cuda_fail(e, "tl pre");
      if ((e = apply3(f[F_U], f[F_R], 1.0, 0)) != cudaSuccess) return cuda_fail(e, "tl rhs");
      // tangent-linear solves stop relative to the increment right-hand side
      if ((e = cudaMemsetAsync(&st->bb, 0, sizeof(double), stream)) != cudaSuccess) return cuda_fail(e, "tl");
      if ((s = pcg()) != RD_OK) return s;
      PwArgs<T> b = pw_args();
      b.a = f[F_CHS];
      b.b = f[F_X];
      b.d = css_slot(n);
      b.out0 = f[F_CH];
      if ((e = L_::pw(kPwTlPost, b, stream)) != cudaSuccess) return cuda_fail(e, "tl post");
    }
    PwArgs<T> a = pw_args();
    a.a = f[F_CH];
    a.out0 = f[F_ALPHA];
    if ((e = L_::pw(kPwNeg, a, stream)) != cudaSuccess) return cuda_fail(e, "negate");
    if ((s = run_adjoint()) != RD_OK) return s;
    s = collect(Hv, v);
    return end_call(s);
  }
};

}  // namespace rd

// ================================================================== C ABI
struct rd_ctx {
  rd::EngineBase* e;
};

static bool valid_config(const rd_config* c) {
  if (!c) return false;
  if (c->nt < 1 || !(c->t_end > 0) || !(c->pcg_rtol > 0) || c->pcg_maxit < 1) return false;
  if (c->prec != RD_FP64 && c->prec != RD_MIXED) return false;
  if (c->ckpt_stride < 0) return false;
  if (c->guess_restart < -1) return false;
  return true;
}
static bool valid_shape(const rd_config* c) {
  for (int a = 0; a < 3; ++a)
    if (!rd::supported_length(c->n[a])) return false;
  return true;
}

namespace {
// Self-test of the bounded mbarrier wait used by every TMA pass: one block
// arms a barrier for 16 bytes of transaction and either issues a 16-byte bulk
// copy that completes it (copy = 1) or issues nothing (copy = 0), then waits
// with `polls` polls.  The outcome (kStOk or kStTimeout) goes to *status.
__global__ void k_selftest_wait(const int4* src, unsigned polls, int copy, int* status) {
  __shared__ alignas(16) int4 buf;
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  rd::mbar_init(&bar, 1);
  rd::fence_barrier_init();
  rd::mbar_expect_tx(&bar, 16);
  if (copy)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];" ::"r"(
            rd::smem_addr(&buf)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(rd::smem_addr(&bar))
        : "memory");
  const bool ok = rd::mbar_wait(&bar, 0, polls);
  *status = !ok ? rd::kStTimeout : (copy && buf.x == src->x && buf.w == src->w) ? rd::kStOk : -1;
}

// Peak fused multiply-add rate: eight independent FMA chains per thread in
// registers, enough warps to fill every scheduler; one value per thread is
// stored so that nothing is optimised away.
template <typename F>
__global__ void __launch_bounds__(256) k_fma_probe(F* out, int iters) {
  F a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = F(threadIdx.x + j) * F(1e-3);
  const F b = F(0.999999), c = F(1e-6);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  F s = F(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
rd_status fma_probe(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RD_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  F* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rd_status st = RD_ERR_CUDA;
  if (cudaMalloc(&out, sizeof(F) * size_t(blocks) * threads) == cudaSuccess &&
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    k_fma_probe<F><<<blocks, threads, 0, s>>>(out, iters);   // warm-up
    cudaEventRecord(e0, s);
    k_fma_probe<F><<<blocks, threads, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      *tflops = 2.0 * 8.0 * iters * double(blocks) * threads / (1e-3 * ms) / 1e12;
      st = RD_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  cudaGetLastError();
  return st;
}

// A field pointer (host or device) must be non-null and aligned to its
// element (FP64): the kernels read caller fields with plain 8-byte loads, and
// a misaligned device address would fault the context instead of failing
// the call.
bool bad_field(const void* p) { return !p || (reinterpret_cast<uintptr_t>(p) & 7u); }
bool bad_opt_field(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 7u); }
// Host parameter vectors must be finite: a NaN weight of a Gaussian would
// otherwise be dropped silently by the basis synthesis, which skips terms
// below its cut-off.
bool bad_vec(const double* v, int n) {
  if (!v) return true;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return true;
  return false;
}
}  // namespace

extern "C" {

rd_status rd_config_default(rd_config* c) {
  if (!c) return RD_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->n[0] = c->n[1] = c->n[2] = 64;
  c->nt = 16;
  c->t_end = 1.0;
  c->prec = RD_FP64;
  c->pcg_rtol = 1e-10;
  c->pcg_maxit = 200;
  c->ckpt_stride = 0;
  c->k_w[0] = 1.0;
  c->k_w[1] = 0.1;
  c->k_w[2] = 0.0;
  c->rho_w[0] = 1.0;
  c->rho_w[1] = 0.2;
  c->rho_w[2] = 0.0;
  c->beta_p = 0.0;
  c->moving_atlas = 0;
  c->coupling = 0;
  c->guess_restart = 0;
  return RD_OK;
}

rd_status rd_workspace_size(const rd_config* cfg, int np, size_t* bytes) {
  if (!valid_config(cfg) || np < 1 || !bytes) return RD_ERR_ARG;
  if (!valid_shape(cfg)) return RD_ERR_SHAPE;
  rd::Carve m{nullptr, 0, 0, true};
  *bytes = (cfg->prec == RD_MIXED) ? rd::Engine<float>::layout(m, *cfg, np, nullptr)
                                   : rd::Engine<double>::layout(m, *cfg, np, nullptr);
  return RD_OK;
}

rd_status rd_create(rd_ctx** out, const rd_config* cfg, int np, void* workspace, size_t workspace_bytes,
                    void* stream) {
  if (!out || !valid_config(cfg) || np < 1) return RD_ERR_ARG;
  if (!valid_shape(cfg)) return RD_ERR_SHAPE;
  *out = nullptr;
  rd_ctx* c = new rd_ctx;
  rd_status s;
  if (cfg->prec == RD_MIXED) {
    auto* e = new rd::Engine<float>();
    c->e = e;
    s = e->init(*cfg, np, workspace, workspace_bytes, (cudaStream_t)stream);
  } else {
    auto* e = new rd::Engine<double>();
    c->e = e;
    s = e->init(*cfg, np, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  if (s != RD_OK) {
    static thread_local char msg[512];
    snprintf(msg, sizeof(msg), "%s", c->e->err);
    delete c->e;
    delete c;
    return s;
  }
  *out = c;
  return RD_OK;
}

rd_status rd_set_tissue(rd_ctx* c, const double* m_wm, const double* m_gm, const double* m_csf) {
  if (!c || bad_field(m_wm) || bad_field(m_gm) || bad_field(m_csf)) return RD_ERR_ARG;
  return c->e->set_tissue(m_wm, m_gm, m_csf);
}

rd_status rd_set_basis(rd_ctx* c, const double* centers, double sigma) {
  if (!c || !centers) return RD_ERR_ARG;
  return c->e->set_basis(centers, sigma);
}

rd_status rd_set_data(rd_ctx* c, const double* d) {
  if (!c || bad_field(d)) return RD_ERR_ARG;
  return c->e->set_data(d);
}

rd_status rd_coupling_field(rd_ctx* c, double* q_wm, double* q_gm, double* q_csf) {
  if (!c || bad_field(q_wm) || bad_field(q_gm) || bad_field(q_csf)) return RD_ERR_ARG;
  return c->e->coupling_field(q_wm, q_gm, q_csf);
}

rd_status rd_forward(rd_ctx* c, const double* p, double k_f, double rho_f, double* c1_out, double* misfit) {
  if (!c || bad_vec(p, c->e->np) || !(k_f >= 0) || !std::isfinite(k_f) || !std::isfinite(rho_f) ||
      bad_opt_field(c1_out))
    return RD_ERR_ARG;
  return c->e->forward(p, k_f, rho_f, c1_out, misfit);
}

rd_status rd_adjoint(rd_ctx* c, double* alpha0_out) {
  if (!c || bad_opt_field(alpha0_out)) return RD_ERR_ARG;
  return c->e->adjoint(alpha0_out);
}

rd_status rd_gradient(rd_ctx* c, const double* p, double k_f, double rho_f, double* misfit, double* grad) {
  if (!c || bad_vec(p, c->e->np) || !grad || !(k_f >= 0) || !std::isfinite(k_f) || !std::isfinite(rho_f))
    return RD_ERR_ARG;
  if (!c->e->have_data) {
    snprintf(c->e->err, sizeof(c->e->err), "rd_set_data is required");
    return RD_ERR_STATE;
  }
  double J = 0.0;
  rd_status s = c->e->forward(p, k_f, rho_f, nullptr, &J);
  if (s != RD_OK && s != RD_ERR_NOCONV) return s;
  const bool nc = (s == RD_ERR_NOCONV);
  s = c->e->adjoint(nullptr);
  if (s != RD_OK && s != RD_ERR_NOCONV) return s;
  if (misfit) *misfit = J;
  for (int i = 0; i < c->e->np + 2; ++i) grad[i] = c->e->last_grad[i];
  return (nc || s == RD_ERR_NOCONV) ? RD_ERR_NOCONV : RD_OK;
}

rd_status rd_last_gradient(const rd_ctx* c, double* grad) {
  if (!c || !grad) return RD_ERR_ARG;
  if (!c->e->have_grad) return RD_ERR_STATE;
  for (int i = 0; i < c->e->np + 2; ++i) grad[i] = c->e->last_grad[i];
  return RD_OK;
}

rd_status rd_hessvec(rd_ctx* c, const double* p, double k_f, double rho_f, const double* v, double* Hv) {
  if (!c || bad_vec(p, c->e->np) || bad_vec(v, c->e->np + 2) || !Hv || !(k_f >= 0) || !std::isfinite(k_f) ||
      !std::isfinite(rho_f))
    return RD_ERR_ARG;
  if (!c->e->have_tissue || !c->e->have_basis) {
    snprintf(c->e->err, sizeof(c->e->err), "rd_set_tissue and rd_set_basis are required");
    return RD_ERR_STATE;
  }
  return c->e->hessvec(p, k_f, rho_f, v, Hv);
}

rd_status rd_apply_operator(rd_ctx* c, double k_f, const double* u, double* Au) {
  if (!c || bad_field(u) || bad_field(Au) || !std::isfinite(k_f)) return RD_ERR_ARG;
  return c->e->apply_operator(k_f, u, Au);
}

rd_status rd_set_precond_scale(rd_ctx* c, double scale) {
  if (!c || !(scale > 0.0) || !std::isfinite(scale)) return RD_ERR_ARG;
  return c->e->set_precond_scale(scale);
}

rd_status rd_apply_precond(rd_ctx* c, double k_f, const double* r, double* z) {
  if (!c || bad_field(r) || bad_field(z) || !(k_f >= 0) || !std::isfinite(k_f)) return RD_ERR_ARG;
  return c->e->apply_precond(k_f, r, z);
}

void rd_profile_enable(int on) {
  rd::Profiler& p = rd::prof();
  std::lock_guard<std::mutex> lk(p.mu);
  p.drain();
  p.on = (on != 0);
  for (int i = 0; i < rd::kcCount; ++i) {
    p.ms[i] = 0.0;
    p.count[i] = 0;
  }
}

int rd_profile_read(double* ms, long long* launches, int n) {
  rd::Profiler& p = rd::prof();
  std::lock_guard<std::mutex> lk(p.mu);
  p.drain();
  for (int i = 0; i < n && i < rd::kcCount; ++i) {
    if (ms) ms[i] = p.ms[i];
    if (launches) launches[i] = p.count[i];
  }
  return rd::kcCount;
}

const char* rd_profile_class(int i) { return (i >= 0 && i < rd::kcCount) ? rd::kClassNames[i] : ""; }

namespace {
// The last batch graph: one branch per context, replayed while the list of
// contexts is unchanged.
struct BatchGraph {
  std::vector<rd_ctx*> ctxs;
  int gen = 0;   // autotuner generation the graph was captured under
  cudaGraphExec_t exec = nullptr;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> events;
  void clear() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto s : branch) cudaStreamDestroy(s);
    for (auto e : events) cudaEventDestroy(e);
    if (origin) cudaStreamDestroy(origin);
    exec = nullptr;
    origin = nullptr;
    branch.clear();
    events.clear();
    ctxs.clear();
  }
};
std::mutex g_batch_mu;
BatchGraph g_batch;
}  // namespace

rd_status rd_set_anatomy_data(rd_ctx* c, const double* md_wm, const double* md_gm, const double* md_csf) {
  if (!c || bad_field(md_wm) || bad_field(md_gm) || bad_field(md_csf)) return RD_ERR_ARG;
  {
    // a batch graph captured before holds misfit launches without m_D
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (std::find(g_batch.ctxs.begin(), g_batch.ctxs.end(), c) != g_batch.ctxs.end()) g_batch.clear();
  }
  return c->e->set_anatomy_data(md_wm, md_gm, md_csf);
}

rd_status rd_batch_gradient(rd_ctx* const* ctxs, int count, const double* const* p, const double* k_f,
                            const double* rho_f, double* misfit, double* const* grad) {
  if (!ctxs || count < 1 || !p || !k_f || !rho_f || !grad) return RD_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || bad_vec(p[i], ctxs[i]->e->np) || !grad[i] || !(k_f[i] >= 0) || !std::isfinite(k_f[i]) ||
        !std::isfinite(rho_f[i]))
      return RD_ERR_ARG;
    rd::EngineBase* e = ctxs[i]->e;
    if (!e->have_tissue || !e->have_basis || !e->have_data) {
      snprintf(e->err, sizeof(e->err), "rd_set_tissue, rd_set_basis and rd_set_data are required");
      return RD_ERR_STATE;
    }
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return RD_ERR_ARG;
  }
  // contexts that have not run yet do one ordinary gradient first (it warms
  // every launcher and leaves the solver state the batch graph expects)
  for (int i = 0; i < count; ++i) {
    rd::EngineBase* e = ctxs[i]->e;
    if (!e->warm()) {
      std::vector<double> gtmp(e->np + 2);
      double J;
      rd_status s = rd_gradient(ctxs[i], p[i], k_f[i], rho_f[i], &J, gtmp.data());
      if (s != RD_OK && s != RD_ERR_NOCONV) return s;
      if (!e->warm()) {
        s = rd_gradient(ctxs[i], p[i], k_f[i], rho_f[i], &J, gtmp.data());
        if (s != RD_OK && s != RD_ERR_NOCONV) return s;
      }
    }
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return RD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  const bool same = (int)g_batch.ctxs.size() == count && g_batch.exec && g_batch.gen == rd::g_tune_gen.load() &&
                    std::equal(g_batch.ctxs.begin(), g_batch.ctxs.end(), ctxs);
  for (int i = 0; i < count; ++i) ctxs[i]->e->batch_prepare(p[i], k_f[i], rho_f[i]);
  if (!same) {
    g_batch.clear();
    BatchGraph& b = g_batch;
    b.gen = rd::g_tune_gen.load();
    b.ctxs.assign(ctxs, ctxs + count);
    cudaError_t ce = cudaStreamCreateWithFlags(&b.origin, cudaStreamNonBlocking);
    b.branch.resize(count, nullptr);
    b.events.resize(count + 1, nullptr);
    for (int i = 0; i < count && ce == cudaSuccess; ++i) ce = cudaStreamCreateWithFlags(&b.branch[i], cudaStreamNonBlocking);
    for (int i = 0; i <= count && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&b.events[i], cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      g_batch.clear();
      return RD_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    rd_status st = RD_OK;
    ce = cudaStreamBeginCapture(b.origin, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) ce = cudaEventRecord(b.events[count], b.origin);
    for (int i = 0; i < count && ce == cudaSuccess && st == RD_OK; ++i) {
      ce = cudaStreamWaitEvent(b.branch[i], b.events[count], 0);
      if (ce == cudaSuccess) st = ctxs[i]->e->batch_enqueue(p[i], k_f[i], rho_f[i], b.branch[i]);
      if (ce == cudaSuccess && st == RD_OK) ce = cudaEventRecord(b.events[i], b.branch[i]);
      if (ce == cudaSuccess && st == RD_OK) ce = cudaStreamWaitEvent(b.origin, b.events[i], 0);
    }
    cudaError_t ee = cudaStreamEndCapture(b.origin, &graph);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess && st == RD_OK) ce = cudaGraphInstantiate(&b.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess || st != RD_OK) {
      cudaGetLastError();
      g_batch.clear();
      if (st == RD_OK) snprintf(ctxs[0]->e->err, sizeof(ctxs[0]->e->err), "batch graph: %s", cudaGetErrorString(ce));
      return st != RD_OK ? st : RD_ERR_CUDA;
    }
    for (int i = 0; i < count; ++i) ctxs[i]->e->batch_prepare(p[i], k_f[i], rho_f[i]);
  }
  cudaError_t ce = cudaGraphLaunch(g_batch.exec, g_batch.origin);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(g_batch.origin);
  if (ce != cudaSuccess) {
    snprintf(ctxs[0]->e->err, sizeof(ctxs[0]->e->err), "batch launch: %s", cudaGetErrorString(ce));
    return RD_ERR_CUDA;
  }
  rd_status worst = RD_OK;
  for (int i = 0; i < count; ++i) {
    rd_status s = ctxs[i]->e->batch_finish(misfit ? &misfit[i] : nullptr, grad[i]);
    if (s != RD_OK && (worst == RD_OK || worst == RD_ERR_NOCONV)) worst = s;
  }
  return worst;
}

rd_status rd_selftest_bounded_wait(unsigned polls, int copy, const void* src16, int* status, void* stream) {
  if (!status || (reinterpret_cast<uintptr_t>(status) & 3u) || polls == 0 || polls > rd::kWaitLimit)
    return RD_ERR_ARG;
  if (copy && (!src16 || (reinterpret_cast<uintptr_t>(src16) & 15u))) return RD_ERR_ARG;
  k_selftest_wait<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const int4*>(copy ? src16 : nullptr), polls, copy, status);
  return cudaGetLastError() == cudaSuccess ? RD_OK : RD_ERR_CUDA;
}

rd_status rd_active_tiles(const rd_ctx* c, long long* counts) {
  if (!c || !counts) return RD_ERR_ARG;
  if (!c->e->have_tissue) return RD_ERR_STATE;
  for (int k = 0; k < 3; ++k) {
    counts[2 * k] = c->e->active_tiles[k];
    counts[2 * k + 1] = c->e->all_tiles[k];
  }
  return RD_OK;
}

rd_status rd_probe_fma_rate(int prec, double* tflops) {
  if (!tflops || (prec != RD_FP64 && prec != RD_MIXED)) return RD_ERR_ARG;
  return prec == RD_FP64 ? fma_probe<double>(tflops) : fma_probe<float>(tflops);
}

int rd_last_pcg_iters(const rd_ctx* c) { return c ? c->e->last_iters : 0; }
int rd_last_graph_solves(const rd_ctx* c) { return c ? c->e->last_graph_solves : 0; }

void rd_autotune_clear(void) { rd::clear_tuned(); }

rd_status rd_autotune(rd_ctx* c, int reps, int* caps, int* pencil, int ncaps) {
  if (!c || reps < 1 || ncaps < 0) return RD_ERR_ARG;
  return c->e->autotune(reps, caps, pencil, ncaps < rd::kcCount ? ncaps : rd::kcCount);
}
int rd_last_pcg_solves(const rd_ctx* c) { return c ? c->e->last_solves : 0; }

const char* rd_last_error(const rd_ctx* c) { return c ? c->e->err : "null context"; }

void rd_destroy(rd_ctx* c) {
  if (!c) return;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (std::find(g_batch.ctxs.begin(), g_batch.ctxs.end(), c) != g_batch.ctxs.end()) g_batch.clear();
  }
  delete c->e;
  delete c;
}

}  // extern "C"
