// Registration engine and its C ABI (include/rg.h): the modified registration
// problem of the Picard iteration (Sec. 2.2, Eq. objective_reg) on the
// device: semi-Lagrangian state and adjoint solves, the Leray-projected
// reduced gradient, the Gauss-Newton Hessian-vector product and the
// spectral preconditioner.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rg.h"
#include "rd_launch_impl.cuh"
#include "rd_reg.cuh"
#include "rd_tables.h"

namespace rd {
namespace {

using namespace reg;

constexpr int kRedBlocks = 512;   // fixed partial count: deterministic sums

struct RegBase {
  virtual ~RegBase() {}
  char err[512] = {0};
  virtual rd_status init() = 0;
  virtual rd_status set_images(const double* const*, const double* const*, const double*, const double* const*) = 0;
  virtual rd_status forward(const double* const*, double* const*, double*) = 0;
  virtual rd_status gradient(const double* const*, double*, double* const*) = 0;
  virtual rd_status hessvec(const double* const*, const double* const*, double* const*) = 0;
  virtual rd_status precond(const double* const*, double* const*) = 0;
  virtual rd_status project(const double* const*, double* const*) = 0;
};

template <typename T>
struct RegEngine final : RegBase {
  using L_ = Launch<T>;
  rg_config cfg;
  Geom g{};
  long long nn = 0;
  cudaStream_t stream = nullptr;
  double h[3] = {0, 0, 0}, h3 = 0;
  std::vector<void*> allocs;
  T *mA[3], *mP[3], *c = nullptr, *q[3];
  T *v[3], *vt[3], *d[3], *dp[3], *D = nullptr, *phi = nullptr, *w1 = nullptr, *w2 = nullptr;
  T *lam[3], *lam2[3], *mt[3], *mt2[3], *s0[3], *s1[3], *b[3], *t3[3], *gf[3];
  V4<T>* pk[1] = {nullptr};   // packed fields for the interpolation gathers
  std::vector<T*> lev;   // (nt + 1) x 3 transported anatomy fields
  double* stage[3];
  double* part = nullptr;
  double* res = nullptr;
  Params* dprm = nullptr;
  PcgState* dst = nullptr;
  cpx<T>* twA[kNumL] = {};
  cpx<T>* twB[kNumL] = {};
  bool have_img = false, have_q = false;

  RegEngine(const rg_config& c_, cudaStream_t s) : cfg(c_), stream(s) {}
  ~RegEngine() override {
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : allocs) cudaFree(p);
  }

  rd_status fail(rd_status s, const char* msg) {
    snprintf(err, sizeof(err), "%s", msg);
    return s;
  }
  rd_status cuda_fail(cudaError_t e, const char* what) {
    snprintf(err, sizeof(err), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return RD_ERR_CUDA;
  }

  template <typename P>
  bool alloc(P** p, size_t bytes) {
    void* q_ = nullptr;
    if (cudaMalloc(&q_, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(q_);
    *p = static_cast<P*>(q_);
    return true;
  }

  rd_status init() override {
    for (int a = 0; a < 3; ++a) {
      g.n[a] = cfg.n[a];
      h[a] = kTwoPiHost / cfg.n[a];
    }
    nn = (long long)cfg.n[0] * cfg.n[1] * cfg.n[2];
    g.nn = nn;
    h3 = h[0] * h[1] * h[2];
    const size_t fb = sizeof(T) * nn;
    bool ok = true;
    T** fields3[] = {mA, mP, q, v, vt, d, dp, lam, lam2, mt, mt2, s0, s1, b, t3, gf};
    for (T** f : fields3)
      for (int k = 0; k < 3; ++k) ok = ok && alloc(&f[k], fb);
    ok = ok && alloc(&c, fb) && alloc(&D, fb) && alloc(&phi, fb) && alloc(&w1, fb) && alloc(&w2, fb);
    ok = ok && alloc(&pk[0], sizeof(V4<T>) * nn);
    lev.assign(size_t(cfg.nt + 1) * 3, nullptr);
    for (auto& p : lev) ok = ok && alloc(&p, fb);
    for (int k = 0; k < 3; ++k) ok = ok && alloc(&stage[k], sizeof(double) * nn);
    ok = ok && alloc(&part, sizeof(double) * kRedBlocks) && alloc(&res, sizeof(double) * 8) &&
         alloc(&dprm, sizeof(Params)) && alloc(&dst, sizeof(PcgState));
    for (int i = 0; i < kNumL && ok; ++i) {
      const int Ls = slot_length(i);
      ok = alloc(&twA[i], sizeof(cpx<T>) * Ls) && alloc(&twB[i], sizeof(cpx<T>) * Ls);
    }
    if (!ok) return fail(RD_ERR_NOMEM, "device memory for the registration context");
    cudaError_t e;
    if ((e = cudaMemsetAsync(dprm, 0, sizeof(Params), stream)) != cudaSuccess) return cuda_fail(e, "init");
    if ((e = cudaMemsetAsync(dst, 0, sizeof(PcgState), stream)) != cudaSuccess) return cuda_fail(e, "init");
    std::vector<cpx<T>> ta, tb;
    for (int i = 0; i < kNumL; ++i) {
      build_twiddles<T>(slot_length(i), ta, tb);
      if ((e = cudaMemcpyAsync(twA[i], ta.data(), sizeof(cpx<T>) * ta.size(), cudaMemcpyHostToDevice, stream)) !=
              cudaSuccess ||
          (e = cudaMemcpyAsync(twB[i], tb.data(), sizeof(cpx<T>) * tb.size(), cudaMemcpyHostToDevice, stream)) !=
              cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "sync");
    }
    return RD_OK;
  }

  // ---------------------------------------------------------- plumbing
  int eblocks(const void* fn) { return detail::grid_for(fn, 0, (nn + kThreads - 1) / kThreads); }

  cudaError_t in1(const double* src, T* dst_, int k) {
    if (is_device_ptr(src)) return L_::from_f64(src, dst_, nn, stream);
    cudaError_t e = cudaMemcpyAsync(stage[k], src, sizeof(double) * nn, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    return L_::from_f64(stage[k], dst_, nn, stream);
  }
  cudaError_t in3(const double* const* src, T* const* dst_) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = in1(src[k], dst_[k], k);
    return e;
  }
  cudaError_t out3(T* const* src, double* const* dst_) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      if (is_device_ptr(dst_[k])) {
        e = L_::to_f64(src[k], dst_[k], nn, 1.0, stream);
      } else {
        e = L_::to_f64(src[k], stage[k], nn, 1.0, stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dst_[k], stage[k], sizeof(double) * nn, cudaMemcpyDeviceToHost, stream);
      }
    }
    return e;
  }

  // out (+)= c (i k~)^order u along `axis`, optionally times w (see DerMode)
  cudaError_t deriv(int mode, int axis, int order, const T* u, const T* w, T* out, double cc) {
    DerivArgs<T> a{};
    a.u = u;
    a.w = w;
    a.out = out;
    a.c = cc;
    a.axis = axis;
    a.order = order;
    a.g = g;
    const int Ln = g.n[axis];
    a.twA = twA[lidx(Ln)];
    a.twB = twB[lidx(Ln)];
    const long long npairs = nn / Ln / 2;
    RD_DISPATCH_L(Ln, {
      constexpr size_t sm = detail::pencil_smem<T, LL>();
      const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
      const bool ct = (axis == 2);
      switch (mode) {
        case kDerSet:
          return ct ? detail::launch_pencil(k_deriv<T, LL, true, kDerSet>, sm, blocks, a, stream)
                    : detail::launch_pencil(k_deriv<T, LL, false, kDerSet>, sm, blocks, a, stream);
        case kDerAdd:
          return ct ? detail::launch_pencil(k_deriv<T, LL, true, kDerAdd>, sm, blocks, a, stream)
                    : detail::launch_pencil(k_deriv<T, LL, false, kDerAdd>, sm, blocks, a, stream);
        default:
          return ct ? detail::launch_pencil(k_deriv<T, LL, true, kDerMulAdd>, sm, blocks, a, stream)
                    : detail::launch_pencil(k_deriv<T, LL, false, kDerMulAdd>, sm, blocks, a, stream);
      }
    })
  }

  // three derivatives along `axis` in one pass (see Deriv3Mode)
  cudaError_t deriv3(int mode, int axis, T* const* u, T* const* w, T* const* out, double cc) {
    Deriv3Args<T> a{};
    for (int k = 0; k < 3; ++k) {
      a.u[k] = u[k];
      a.w[k] = w[k];
      a.out[k] = out[k];
    }
    a.c = cc;
    a.axis = axis;
    a.g = g;
    const int Ln = g.n[axis];
    a.twA = twA[lidx(Ln)];
    a.twB = twB[lidx(Ln)];
    const long long npairs = nn / Ln / 2;
    RD_DISPATCH_L(Ln, {
      constexpr size_t sm = detail::pencil_smem<T, LL>();
      const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
      const bool ct = (axis == 2);
      if (mode == kD3Body)
        return ct ? detail::launch_pencil(k_deriv3<T, LL, true, kD3Body>, sm, blocks, a, stream)
                  : detail::launch_pencil(k_deriv3<T, LL, false, kD3Body>, sm, blocks, a, stream);
      return ct ? detail::launch_pencil(k_deriv3<T, LL, true, kD3Src>, sm, blocks, a, stream)
                : detail::launch_pencil(k_deriv3<T, LL, false, kD3Src>, sm, blocks, a, stream);
    })
  }

  cudaError_t hartley(int axis, const T* in, T* out) {
    DhtArgs<T> a{};
    a.in = in;
    a.out = out;
    a.axis = axis;
    a.g = g;
    a.twA = twA[lidx(g.n[axis])];
    a.twB = twB[lidx(g.n[axis])];
    a.prm = dprm;
    a.st = dst;
    return L_::dht(g.n[axis], kDhtPlain, a, stream);
  }

  // out = F^-1 S F in with S = inn / (a1 |k~|^2), inn * z0 where |k~|^2 = 0
  // (separable Hartley passes along axes 2 and 1 around the axis-0 pass)
  cudaError_t solve(const T* in, T* out, double a1, double z0, double inn) {
    cudaError_t e;
    if ((e = hartley(2, in, w1)) != cudaSuccess) return e;
    if ((e = hartley(1, w1, w2)) != cudaSuccess) return e;
    SolveArgs<T> a{};
    a.in = w2;
    a.out = w1;
    a.g = g;
    a.twA = twA[lidx(g.n[0])];
    a.twB = twB[lidx(g.n[0])];
    a.a1 = a1;
    a.z0 = z0;
    a.inn = inn;
    const int L0 = g.n[0];
    const long long npairs = nn / L0 / 2;
    RD_DISPATCH_L(L0, {
      constexpr size_t sm = detail::pencil_smem<T, LL>();
      const long long blocks = (npairs + Shape<LL>::G - 1) / Shape<LL>::G;
      e = detail::launch_pencil(k_solve0<T, LL>, sm, blocks, a, stream);
      break;
    })
    if (e != cudaSuccess) return e;
    if ((e = hartley(1, w1, w2)) != cudaSuccess) return e;
    return hartley(2, w2, out);
  }

  cudaError_t div(T* const* w, T* out) {
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = deriv(a == 0 ? kDerSet : kDerAdd, a, 1, w[a], nullptr, out, 1.0);
    return e;
  }

  // out = K w = w - grad phi, -Lap phi = -div w (out may alias w)
  cudaError_t leray(T* const* w, T* const* out) {
    cudaError_t e;
    if ((e = div(w, D)) != cudaSuccess) return e;
    if ((e = solve(D, phi, 1.0, 0.0, -1.0 / double(nn))) != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a) {
      if (out[a] != w[a] &&
          (e = cudaMemcpyAsync(out[a], w[a], sizeof(T) * nn, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
        return e;
      if ((e = deriv(kDerAdd, a, 1, phi, nullptr, out[a], -1.0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // out (+)= coef (-Lap) u per component
  cudaError_t neg_lap(T* const* u, T* const* out, double coef, bool add) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3 && e == cudaSuccess; ++a)
        e = deriv((a == 0 && !add) ? kDerSet : kDerAdd, a, 2, u[k], nullptr, out[k], -coef);
    return e;
  }

  cudaError_t pack4(const T* x, const T* y, const T* z, const T* w, V4<T>* out) {
    k_pack4<T><<<eblocks(reinterpret_cast<const void*>(k_pack4<T>)), kThreads, 0, stream>>>(x, y, z, w, out, nn);
    return cudaGetLastError();
  }

  cudaError_t feet(const T* const* vel, T* const* out, double sign) {
    cudaError_t e = pack4(vel[0], vel[1], vel[2], nullptr, pk[0]);
    if (e != cudaSuccess) return e;
    FeetArgs<T> a{};
    a.vp = pk[0];
    for (int k = 0; k < 3; ++k) {
      a.v[k] = vel[k];
      a.d[k] = out[k];
      a.cdt[k] = T(sign / double(cfg.nt) / h[k]);
    }
    a.g = g;
    k_feet<T><<<eblocks(reinterpret_cast<const void*>(k_feet<T>)), kThreads, 0, stream>>>(a);
    return cudaGetLastError();
  }

  template <int MODE>
  cudaError_t interp_step(const InterpArgs<T>& a0) {
    InterpArgs<T> a = a0;
    if (MODE != kIpInc) {
      const cudaError_t e = pack4(a.u[0], a.u[1], a.u[2], MODE == kIpAdj ? a.D : nullptr, pk[0]);
      if (e != cudaSuccess) return e;
      a.pk[0] = pk[0];
    }
    k_interp<T, MODE><<<eblocks(reinterpret_cast<const void*>(k_interp<T, MODE>)), kThreads, 0, stream>>>(a);
    return cudaGetLastError();
  }

  T* L3(int j, int k) { return lev[size_t(j) * 3 + k]; }

  // m^0 = m_A, m^{j+1} = m^j(X); feet d for the state, dp for the adjoint
  cudaError_t run_forward() {
    cudaError_t e;
    if ((e = feet(v, d, -1.0)) != cudaSuccess) return e;
    for (int k = 0; k < 3; ++k)
      if ((e = cudaMemcpyAsync(L3(0, k), mA[k], sizeof(T) * nn, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
        return e;
    InterpArgs<T> a{};
    a.g = g;
    a.dt = T(1.0 / cfg.nt);
    for (int k = 0; k < 3; ++k) a.d[k] = d[k];
    for (int j = 0; j < cfg.nt; ++j) {
      for (int k = 0; k < 3; ++k) {
        a.u[k] = L3(j, k);
        a.out[k] = L3(j + 1, k);
      }
      if ((e = interp_step<kIpPlain>(a)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  cudaError_t sum_parts(int slot) {
    k_sum_parts<<<1, kThreads, 0, stream>>>(part, kRedBlocks, res + slot);
    return cudaGetLastError();
  }

  // res[0] = misfit sums, res[1] = <v, -Lap v>; lam = l(1); t3 = -Lap v
  cudaError_t objective_and_final() {
    cudaError_t e;
    FinalArgs<T> f{};
    for (int k = 0; k < 3; ++k) {
      f.m[k] = L3(cfg.nt, k);
      f.mp[k] = mP[k];
      f.q[k] = have_q ? q[k] : nullptr;
      f.lam[k] = lam[k];
    }
    f.c = c;
    f.part = part;
    f.nn = nn;
    k_final<T, kFinalState><<<kRedBlocks, kThreads, 0, stream>>>(f);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = sum_parts(0)) != cudaSuccess) return e;
    if ((e = neg_lap(v, t3, 1.0, false)) != cudaSuccess) return e;
    DotArgs<T> da{};
    for (int k = 0; k < 3; ++k) {
      da.x[k] = v[k];
      da.y[k] = t3[k];
    }
    da.part = part;
    da.nn = nn;
    k_dot3<T><<<kRedBlocks, kThreads, 0, stream>>>(da);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sum_parts(1);
  }

  rd_status read_J(double* J) {
    double hr[2];
    cudaError_t e = cudaMemcpyAsync(hr, res, sizeof(hr), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "read objective");
    if (J) *J = h3 * hr[0] + 0.5 * cfg.beta_v * h3 * hr[1];
    if (!std::isfinite(hr[0]) || !std::isfinite(hr[1])) return fail(RD_ERR_NONFINITE, "non-finite objective");
    return RD_OK;
  }

  // From l(1) in lam: the adjoint sweep and b = int sum_i l_i grad m_i dt
  // (trapezoidal in time); the result K[b] in out.
  cudaError_t adjoint_body(T* const* out) {
    cudaError_t e;
    if ((e = feet(v, dp, +1.0)) != cudaSuccess) return e;
    if ((e = div(v, D)) != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a)
      if ((e = cudaMemsetAsync(b[a], 0, sizeof(T) * nn, stream)) != cudaSuccess) return e;
    const double dt = 1.0 / cfg.nt;
    InterpArgs<T> ia{};
    ia.g = g;
    ia.dt = T(dt);
    ia.D = D;
    for (int k = 0; k < 3; ++k) ia.d[k] = dp[k];
    for (int j = cfg.nt; j >= 0; --j) {
      if (j < cfg.nt) {
        for (int k = 0; k < 3; ++k) {
          ia.u[k] = lam[k];
          ia.out[k] = lam2[k];
        }
        if ((e = interp_step<kIpAdj>(ia)) != cudaSuccess) return e;
        for (int k = 0; k < 3; ++k) std::swap(lam[k], lam2[k]);
      }
      const double wj = dt * ((j == 0 || j == cfg.nt) ? 0.5 : 1.0);
      T* mj[3] = {L3(j, 0), L3(j, 1), L3(j, 2)};
      for (int a = 0; a < 3; ++a) {
        T* ba[3] = {b[a], b[a], b[a]};
        if ((e = deriv3(kD3Body, a, mj, lam, ba, wj)) != cudaSuccess) return e;
      }
    }
    return leray(b, out);
  }

  rd_status end(cudaError_t e, const char* what) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return RD_OK;
  }

  // ------------------------------------------------------------ API
  rd_status set_images(const double* const* ma, const double* const* mp, const double* c1,
                       const double* const* qq) override {
    cudaError_t e = in3(ma, mA);
    if (e == cudaSuccess) e = in3(mp, mP);
    if (e == cudaSuccess) e = in1(c1, c, 0);
    have_q = (qq != nullptr);
    if (e == cudaSuccess && have_q) e = in3(qq, q);
    rd_status s = end(e, "set images");
    if (s == RD_OK) have_img = true;
    return s;
  }

  rd_status forward(const double* const* vin, double* const* m1, double* J) override {
    if (!have_img) return fail(RD_ERR_STATE, "rg_set_images is required");
    cudaError_t e = in3(vin, v);
    if (e == cudaSuccess) e = run_forward();
    if (e == cudaSuccess) e = objective_and_final();
    if (e == cudaSuccess && m1) {
      T* last[3] = {L3(cfg.nt, 0), L3(cfg.nt, 1), L3(cfg.nt, 2)};
      e = out3(last, m1);
    }
    rd_status s = end(e, "forward");
    if (s != RD_OK) return s;
    return read_J(J);
  }

  rd_status gradient(const double* const* vin, double* J, double* const* gout) override {
    if (!have_img) return fail(RD_ERR_STATE, "rg_set_images is required");
    cudaError_t e = in3(vin, v);
    if (e == cudaSuccess) e = run_forward();
    if (e == cudaSuccess) e = objective_and_final();
    if (e == cudaSuccess) e = adjoint_body(gf);
    if (e == cudaSuccess) e = neg_lap(v, gf, cfg.beta_v, true);
    if (e == cudaSuccess) e = out3(gf, gout);
    rd_status s = end(e, "gradient");
    if (s != RD_OK) return s;
    return read_J(J);
  }

  // s_k = grad(m_k^j) . vt
  cudaError_t source(int j, T* const* s) {
    cudaError_t e;
    for (int k = 0; k < 3; ++k)
      if ((e = cudaMemsetAsync(s[k], 0, sizeof(T) * nn, stream)) != cudaSuccess) return e;
    T* mj[3] = {L3(j, 0), L3(j, 1), L3(j, 2)};
    for (int a = 0; a < 3; ++a) {
      T* wa[3] = {vt[a], vt[a], vt[a]};
      if ((e = deriv3(kD3Src, a, mj, wa, s, 1.0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  rd_status hessvec(const double* const* vin, const double* const* vtin, double* const* hv) override {
    if (!have_img) return fail(RD_ERR_STATE, "rg_set_images is required");
    cudaError_t e = in3(vin, v);
    if (e == cudaSuccess) e = in3(vtin, vt);
    if (e == cudaSuccess) e = run_forward();
    // incremental state: m~^{j+1} = m~^j(X) - dt/2 (s^j(X) + s^{j+1}(x))
    if (e == cudaSuccess) e = source(0, s0);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemsetAsync(mt[k], 0, sizeof(T) * nn, stream);
    InterpArgs<T> ia{};
    ia.g = g;
    ia.dt = T(1.0 / cfg.nt);
    for (int k = 0; k < 3; ++k) ia.d[k] = d[k];
    for (int j = 0; j < cfg.nt && e == cudaSuccess; ++j) {
      e = source(j + 1, s1);
      for (int k = 0; k < 3; ++k) {
        ia.u[k] = mt[k];
        ia.s[k] = s0[k];
        ia.s1[k] = s1[k];
        ia.out[k] = mt2[k];
      }
      if (e == cudaSuccess) e = interp_step<kIpInc>(ia);
      for (int k = 0; k < 3; ++k) {
        std::swap(mt[k], mt2[k]);
        std::swap(s0[k], s1[k]);
      }
    }
    if (e == cudaSuccess) {
      FinalArgs<T> f{};
      for (int k = 0; k < 3; ++k) {
        f.m[k] = mt[k];
        f.lam[k] = lam[k];
      }
      f.c = c;
      f.nn = nn;
      k_final<T, kFinalInc><<<eblocks(reinterpret_cast<const void*>(k_final<T, kFinalInc>)), kThreads, 0, stream>>>(f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = adjoint_body(gf);
    if (e == cudaSuccess) e = neg_lap(vt, gf, cfg.beta_v, true);
    if (e == cudaSuccess) e = out3(gf, hv);
    return end(e, "hessvec");
  }

  rd_status precond(const double* const* r, double* const* z) override {
    cudaError_t e = in3(r, gf);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
      e = solve(gf[k], t3[k], cfg.beta_v, 1.0 / cfg.beta_v, 1.0 / double(nn));
    if (e == cudaSuccess) e = out3(t3, z);
    return end(e, "precond");
  }

  rd_status project(const double* const* w, double* const* kw) override {
    cudaError_t e = in3(w, gf);
    if (e == cudaSuccess) e = leray(gf, gf);
    if (e == cudaSuccess) e = out3(gf, kw);
    return end(e, "project");
  }
};

bool supported(int L) {
  return L == 8 || L == 16 || L == 32 || L == 64 || L == 96 || L == 128 || L == 256;
}

}  // namespace
}  // namespace rd

struct rg_ctx {
  rd::RegBase* e;
};

namespace {
// Field pointers (host or device) must be non-null and 8-byte aligned: the
// kernels read them with plain FP64 loads.
bool bad3(const double* const* f) {
  if (!f) return true;
  for (int k = 0; k < 3; ++k)
    if (!f[k] || (reinterpret_cast<uintptr_t>(f[k]) & 7u)) return true;
  return false;
}
bool bad1(const void* p) { return !p || (reinterpret_cast<uintptr_t>(p) & 7u); }
}  // namespace

extern "C" {

rd_status rg_config_default(rg_config* cfg) {
  if (!cfg) return RD_ERR_ARG;
  cfg->n[0] = cfg->n[1] = cfg->n[2] = 64;
  cfg->nt = 8;
  cfg->prec = RD_FP64;
  cfg->beta_v = 1e-2;
  return RD_OK;
}

rd_status rg_create(rg_ctx** out, const rg_config* cfg, void* stream) {
  if (!out || !cfg) return RD_ERR_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!rd::supported(cfg->n[a])) return RD_ERR_SHAPE;
  if (cfg->nt < 1 || !(cfg->beta_v > 0) || (cfg->prec != RD_FP64 && cfg->prec != RD_MIXED)) return RD_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rd::RegBase* e = (cfg->prec == RD_FP64) ? static_cast<rd::RegBase*>(new rd::RegEngine<double>(*cfg, s))
                                          : static_cast<rd::RegBase*>(new rd::RegEngine<float>(*cfg, s));
  rd_status st = e->init();
  if (st != RD_OK) {
    delete e;
    return st;
  }
  *out = new rg_ctx{e};
  return RD_OK;
}

rd_status rg_set_images(rg_ctx* c, const double* const* ma, const double* const* mp, const double* c1,
                        const double* const* q) {
  if (!c || bad3(ma) || bad3(mp) || bad1(c1) || (q && bad3(q))) return RD_ERR_ARG;
  return c->e->set_images(ma, mp, c1, q);
}

rd_status rg_forward(rg_ctx* c, const double* const* v, double* const* m1, double* J) {
  if (!c || bad3(v) || (m1 && bad3(m1))) return RD_ERR_ARG;
  return c->e->forward(v, m1, J);
}

rd_status rg_gradient(rg_ctx* c, const double* const* v, double* J, double* const* g) {
  if (!c || bad3(v) || bad3(g)) return RD_ERR_ARG;
  return c->e->gradient(v, J, g);
}

rd_status rg_hessvec(rg_ctx* c, const double* const* v, const double* const* vt, double* const* hv) {
  if (!c || bad3(v) || bad3(vt) || bad3(hv)) return RD_ERR_ARG;
  return c->e->hessvec(v, vt, hv);
}

rd_status rg_apply_precond(rg_ctx* c, const double* const* r, double* const* z) {
  if (!c || bad3(r) || bad3(z)) return RD_ERR_ARG;
  return c->e->precond(r, z);
}

rd_status rg_project(rg_ctx* c, const double* const* w, double* const* kw) {
  if (!c || bad3(w) || bad3(kw)) return RD_ERR_ARG;
  return c->e->project(w, kw);
}

const char* rg_last_error(const rg_ctx* c) { return c ? c->e->err : ""; }

rd_status rg_destroy(rg_ctx* c) {
  if (!c) return RD_ERR_ARG;
  delete c->e;
  delete c;
  return RD_OK;
}

}  // extern "C"
