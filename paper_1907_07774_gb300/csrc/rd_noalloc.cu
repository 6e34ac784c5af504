// Allocation-free variant of the spectral preconditioner application.
//
// Some callers cannot allocate device memory at the point where they need
// the preconditioner: applications whose device memory is entirely owned by
// another framework's pool (so cudaMalloc either fails or fragments that
// pool), and latency-critical loops that must not pay cudaMalloc/cudaFree's
// implicit device synchronisation.  rd_apply_precond_static serves them: it
// takes the caller's input and output buffers and keeps every other byte it
// needs (solver scalars, FP64 reduction partials and their completion counter,
// FFT twiddle tables) in one file-scope __device__ array, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array is a fixed 128 KiB that every GPU loading this library holds
// until process exit.  All calls share it and it keeps the previous call's
// contents: each call first runs a one-block kernel on the caller's stream
// that rewrites the scalars, clears the solver state and clears the reduction
// counters, so nothing of an earlier call is read.  Calls that overlap on the
// GPU (different streams, or different host threads without ordering) race on
// this array.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/rd.h"
#include "rd_launch.cuh"
#include "rd_tables.h"

namespace rd {
namespace {

constexpr int kNumLengths = 7;   // pencil lengths 8, 16, ..., 256 and 96
constexpr int kMaxLength = 256;
constexpr int kMaxDevices = 64;

// Every member starts on a 256-byte boundary (the twiddle tables are read
// with 16-byte vector loads).
struct StaticScratch {
  alignas(256) Params prm;
  alignas(256) PcgState st;
  alignas(256) unsigned int counter[64];
  alignas(256) double part[kMaxBlocks];
  alignas(256) cpx<double> twA[kNumLengths][kMaxLength];
  alignas(256) cpx<double> twB[kNumLengths][kMaxLength];
};
static_assert(offsetof(StaticScratch, twA) % 256 == 0 && offsetof(StaticScratch, twB) % 256 == 0,
              "twiddle tables must be 256-byte aligned");

constexpr size_t kScratchBytes = 128 * 1024;   // fits StaticScratch (about 100 KiB)
static_assert(sizeof(StaticScratch) <= kScratchBytes, "static scratch too small");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSlot {
  bool ready = false;
  StaticScratch* ptr = nullptr;   // device address of g_scratch on that device
};
std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

int length_index(int L) { return lidx(L); }

// Start of a call: this call's scalars (passed by value, so no host buffer
// is read by a copy), a cleared solver state and cleared counters.
__global__ void k_static_begin(StaticScratch* d, Params prm) {
  const int t = threadIdx.x;
  if (t == 0) {
    d->prm = prm;
    memset(&d->st, 0, sizeof(PcgState));
  }
  if (t < 64) d->counter[t] = 0u;
}

// Once per device, with that device current: find the array's device
// address (the host-side symbol is only a stand-in) and upload the twiddle
// tables computed in FP64 on the host.
rd_status setup_device(int dev, StaticScratch** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSlot& s = g_slots[dev];
  if (s.ready) {
    *out = s.ptr;
    return RD_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return RD_ERR_CUDA;
  }
  StaticScratch* d = reinterpret_cast<StaticScratch*>(p);
  std::vector<cpx<double>> ta, tb;
  for (int i = 0; i < kNumLengths; ++i) {
    const int L = slot_length(i);
    build_twiddles<double>(L, ta, tb);
    ta.resize(kMaxLength, cpx<double>{0.0, 0.0});
    tb.resize(kMaxLength, cpx<double>{0.0, 0.0});
    if (cudaMemcpy(&d->twA[i][0], ta.data(), sizeof(cpx<double>) * kMaxLength, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(&d->twB[i][0], tb.data(), sizeof(cpx<double>) * kMaxLength, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      return RD_ERR_CUDA;
    }
  }
  // A copy from pageable host memory may return before the data reach the
  // device, and it is ordered only with the legacy default stream; the
  // caller's stream may be a non-blocking one.  Wait for the tables here.
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return RD_ERR_CUDA;
  }
  s.ptr = d;
  s.ready = true;
  *out = d;
  return RD_OK;
}

}  // namespace
}  // namespace rd

extern "C" rd_status rd_apply_precond_static(const int n[3], double coef, const double* r, double* z,
                                             void* stream) {
  using namespace rd;
  if (!n || !r || !z || !std::isfinite(coef) || coef < 0.0) return RD_ERR_ARG;
  // the pencil kernels read and write pairs of values with 16-byte accesses
  if ((reinterpret_cast<uintptr_t>(r) & 15) || (reinterpret_cast<uintptr_t>(z) & 15)) return RD_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!supported_length(n[a]) || n[a] > kMaxLength) return RD_ERR_SHAPE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RD_ERR_CUDA;
  StaticScratch* d = nullptr;
  rd_status s = setup_device(dev, &d);
  if (s != RD_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Geom g;
  for (int a = 0; a < 3; ++a) g.n[a] = n[a];
  g.nn = (long long)n[0] * n[1] * n[2];
  // scalars of this call (s = k_f-free symbol: coef = tau/2 k_f mean(kappa1))
  Params prm;
  memset(&prm, 0, sizeof(prm));
  prm.s = 1.0;
  prm.k_f = coef;
  prm.kbar1 = 1.0;
  prm.inv_nn = 1.0 / double(g.nn);
  k_static_begin<<<1, 64, 0, st>>>(d, prm);
  if (cudaGetLastError() != cudaSuccess) return RD_ERR_CUDA;
  auto args = [&](int axis, const double* in, double* out) {
    DhtArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.axis = axis;
    a.g = g;
    a.twA = d->twA[length_index(n[axis])];
    a.twB = d->twB[length_index(n[axis])];
    a.prm = &d->prm;
    a.st = &d->st;
    a.fin.kind = kFinRz;
    a.fin.st = &d->st;
    a.fin.prm = &d->prm;
    a.fin.part = d->part;
    a.fin.counter = &d->counter[0];
    return a;
  };
  // Hartley passes x, y, (z S z), y, x; everything after the first pass works
  // in place on the caller's output.
  cudaError_t e;
  if ((e = Launch<double>::dht(n[2], kDhtPlain, args(2, r, z), st)) != cudaSuccess ||
      (e = Launch<double>::dht(n[1], kDhtPlain, args(1, z, z), st)) != cudaSuccess ||
      (e = Launch<double>::dht(n[0], kDhtSym, args(0, z, z), st)) != cudaSuccess ||
      (e = Launch<double>::dht(n[1], kDhtPlain, args(1, z, z), st)) != cudaSuccess ||
      (e = Launch<double>::dht(n[2], kDhtPlain, args(2, z, z), st)) != cudaSuccess) {
    cudaGetLastError();
    return RD_ERR_CUDA;
  }
  return RD_OK;
}
