/*
 * C ABI of the registration sub-problem of the Picard iteration (arXiv
 * 1907.07774, Sec. 2.2, Eq. objective_reg): for a fixed tumor c(1) and
 * coupling field q, find the stationary velocity v that transports the atlas
 * anatomy m_A onto the patient anatomy m_P:
 *
 *   J(v) = 1/2 h^3 sum_i sum_x (m_i(1) (1 - c) - m_P,i)^2 + h^3 sum_x q . m(1)
 *          + beta_v / 2 |grad v|^2                          (Eq. registr_reg)
 *   dm/dt + grad(m) v = 0,  m(0) = m_A                      (Eq. reg:fwd)
 *
 * with the adjoint -dl/dt - div(l v) = 0 (Eq. reg:adj), the reduced gradient
 * beta_v (-Lap) v + K[int_0^1 sum_i l_i grad m_i dt] (Eq. reg:inv), K the
 * Leray projection onto divergence-free fields (div v = w with w = 0), and
 * the Gauss-Newton Hessian-vector product.  Discretisation (Sec. 3.3):
 * semi-Lagrangian steps dt = 1 / nt along Heun characteristic feet with
 * periodic tricubic Lagrange interpolation; spectral derivatives (Nyquist
 * symbol of first derivatives zeroed) on the periodic grid [0, 2 pi)^3.
 *
 * Fields: FP64, n0 * n1 * n2 values, C order (index 2 fastest), in host or
 * device memory (unified addressing decides); a vector field is an array of
 * three such pointers (components along axes 0, 1, 2).  The caller owns all
 * buffers; the context owns its device memory.  Every call is synchronous
 * on the context's stream.  Status codes and rd_status are those of rd.h.
 */
#ifndef RG_H
#define RG_H

#include "rd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rg_ctx rg_ctx;

typedef struct rg_config {
  int n[3];       /* grid; each a supported pencil length (rd.h) */
  int nt;         /* semi-Lagrangian steps on [0, 1], >= 1 */
  int prec;       /* RD_FP64 or RD_MIXED (FP32 fields, FP64 reductions) */
  double beta_v;  /* weight of the H^1 seminorm, > 0 */
} rg_config;

/* Defaults: 64^3, nt = 8, FP64, beta_v = 1e-2. */
rd_status rg_config_default(rg_config* cfg);

/* Creates a context on `stream` (a cudaStream_t, or NULL for the legacy
 * default stream).  RD_ERR_SHAPE for unsupported sizes, RD_ERR_ARG for other
 * out-of-range parameters, RD_ERR_NOMEM if device memory cannot be
 * allocated. */
rd_status rg_create(rg_ctx** out, const rg_config* cfg, void* stream);

/* Atlas anatomy m_A, patient anatomy m_P (three fields each), tumor c(1)
 * and the coupling field q (three fields, or NULL for q = 0). */
rd_status rg_set_images(rg_ctx* ctx, const double* const* m_atlas, const double* const* m_patient,
                        const double* c1, const double* const* q);

/* State solve: J(v) and optionally m(1) (three fields, or NULL).
 * RD_ERR_STATE before rg_set_images. */
rd_status rg_forward(rg_ctx* ctx, const double* const* v, double* const* m1_out, double* J);

/* J(v) and the reduced gradient g (three fields). */
rd_status rg_gradient(rg_ctx* ctx, const double* const* v, double* J, double* const* g);

/* Gauss-Newton Hessian-vector product at v in direction vt. */
rd_status rg_hessvec(rg_ctx* ctx, const double* const* v, const double* const* vt, double* const* hv);

/* z = (beta_v (-Lap))^-1 r per component, the zero mode divided by beta_v
 * (the preconditioner of the Gauss-Newton-Krylov solve, Sec. 3.2). */
rd_status rg_apply_precond(rg_ctx* ctx, const double* const* r, double* const* z);

/* kw = K w, the Leray projection onto divergence-free fields. */
rd_status rg_project(rg_ctx* ctx, const double* const* w, double* const* kw);

/* Message of the last failed call ("" if none). */
const char* rg_last_error(const rg_ctx* ctx);

rd_status rg_destroy(rg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RG_H */
