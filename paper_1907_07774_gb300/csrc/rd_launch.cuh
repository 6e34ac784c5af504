// Host launchers for the kernels of rd_passes.cuh, one explicit
// instantiation per working precision (rd_kern_f32.cu, rd_kern_f64.cu).
#pragma once

#include "rd_tma.cuh"

namespace rd {

constexpr int kMaxBlocks = 4096;   // capacity of the reduction partial buffer

bool supported_length(int L);

// Kernel classes for the optional per-launch event timing.
enum KClass {
  kcOpContig = 0, kcOpStrided, kcPcgOpx, kcDhtSetup, kcDhtPlain, kcDhtUpdate, kcDhtSym,
  kcGrad, kcPointwise, kcOther, kcCount
};
// When timing is on, every launch is bracketed by two CUDA events on its
// stream; prof_begin returns a token for prof_end (-1 when off).
int prof_begin(int cls, cudaStream_t s);
bool prof_active();
// Choices made by the autotuner, per kernel class and pencil length L:
// the persistent grid size (0: none, the launcher then uses every block that
// fits on the device) and the tile shape (false: the TMA tile kernel, i.e.
// 64-byte column tiles or whole-row tiles staged in shared memory; true: the
// pencil kernel, i.e. 256-thread blocks of TH-lane pencil groups with direct
// loads and stores).
int tuned_cap(int cls, int L);
bool tuned_pencil(int cls, int L);
void set_tuned(int cls, int L, int cap, bool pencil);
void clear_tuned();
// Tensor map for TMA tiles of a strided pass: box {64 B of i2, L along the
// axis}, 64-byte swizzle.  Cached per (pointer, grid, element size, axis);
// false if the map cannot be made (the caller then uses the direct kernels).
bool strided_map(CUtensorMap* out, const void* ptr, const Geom& g, int esz, int axis);
// Tensor map over the [n0 n1][n2] row view: box {n2, rows}, no swizzle.
bool row_map(CUtensorMap* out, const void* ptr, const Geom& g, int esz, int rows);
void prof_end(int token, cudaStream_t s);

template <typename T>
struct Launch {
  static cudaError_t op(int L, const OpArgs<T>& a, cudaStream_t s);
  static cudaError_t dht(int L, int mode, const DhtArgs<T>& a, cudaStream_t s);
  static cudaError_t pcg_opx(int L, const PcgOpxArgs<T>& a, cudaStream_t s);
  static cudaError_t grad(int L, const GradArgs<T>& a, cudaStream_t s);
  static cudaError_t pw(int kind, const PwArgs<T>& a, cudaStream_t s);
  static cudaError_t coef(const CoefArgs<T>& a, cudaStream_t s);
  static cudaError_t phi(const PhiArgs<T>& a, cudaStream_t s);
  static cudaError_t phit(const PhiArgs<T>& a, double* out, double scale, cudaStream_t s);
  static cudaError_t from_f64(const double* in, T* out, long long nn, cudaStream_t s);
  static cudaError_t to_f64(const T* in, double* out, long long nn, double scale, cudaStream_t s);
  static cudaError_t combine(const T* qk, const T* qr, double ca, double cb, double* out, long long nn,
                             cudaStream_t s);
  static cudaError_t normsq(const NormArgs<T>& a, cudaStream_t s);
  static cudaError_t cg_final(T* x, const T* p, const PcgState* st, long long nn, cudaStream_t s);
  static cudaError_t x_init(T* x, const PcgState* st, long long nn, cudaStream_t s);
  static cudaError_t guess(T* r, T* x, T* fs, const T* d1, const T* d2, const T* g1, const T* g2, int order,
                           long long nn, cudaStream_t s);
  static cudaError_t guess_keep(T* d, T* g, const T* x, const T* r, const T* fs, long long nn, cudaStream_t s);
};

extern template struct Launch<float>;
extern template struct Launch<double>;

}  // namespace rd
