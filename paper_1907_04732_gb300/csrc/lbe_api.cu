// C ABI of the LBE library (declarations and contracts in include/lbe.h).
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "lbe_internal.cuh"

using lbe::Geo;
using lbe::Phys;

namespace {

const char *g_static_err = "invalid handle";
thread_local std::string g_thread_err;

int fail(lbe_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  return code;
}

#define LBE_CK(h, expr)                                                                      \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((h), LBE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
  } while (0)

// When the caller passes no stream the library works on a private stream and
// finishes every call with a synchronisation, so that results are complete
// when the call returns.
struct StreamGuard {
  lbe_handle *h;
  bool own;
  ~StreamGuard() {
    if (own && h && h->stream) cudaStreamSynchronize(h->stream);
  }
};

bool fp32(const lbe_handle *h) { return h->prm.precision == LBE_FP32; }

void free_all(lbe_handle *h) {
  void *ptrs[] = {h->id, h->mask, h->f[0], h->f[1], h->n, h->nstar, h->phi, h->u, h->qpart, h->qout, h->psi_dev,
                  h->f32[0], h->f32[1], h->q, h->qstar, h->phifx, h->phi32, h->u32, h->flag, h->lf};
  for (void *p : ptrs) cudaFree(p);
  if (h->qhost) cudaFreeHost(h->qhost);
  lbe::poisson_free(h);
  lbe::mg_free(h);
  lbe::adjoint_free(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
}

// next event of the profiling pool (grown on demand)
cudaError_t next_event(lbe_handle *h, cudaEvent_t *ev) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->ev_pool.push_back(e);
  }
  *ev = h->ev_pool[h->ev_used++];
  return cudaSuccess;
}

cudaError_t mark(lbe_handle *h) {
  if (!h->profiling) return cudaSuccess;
  cudaEvent_t e;
  cudaError_t err = next_event(h, &e);
  if (err != cudaSuccess) return err;
  return cudaEventRecord(e, h->stream);
}

}  // namespace

namespace lbe {
void set_static_error(const char *msg) { g_thread_err = msg; }

void fill_constants(lbe_handle *h) {
  const lbe_params *p = &h->prm;
  Phys &P = h->phys;
  memset(&P, 0, sizeof(P));
  const double A0 = 1.0 + 2.0 * sqrt(2.0);
  P.ns = p->nspecies;
  for (int k = 0; k < p->nspecies; ++k) {
    P.z[k] = p->z[k];
    P.d[k] = p->D[k] / A0;
    P.inv_d[k] = p->D[k] > 0.0 ? A0 / p->D[k] : 0.0;
  }
  for (int i = 0; i < lbe::kQ; ++i)
    P.e_dot_c[i] = p->e_app[0] * lbe::cx_of(i) + p->e_app[1] * lbe::cy_of(i) + p->e_app[2] * lbe::cz_of(i);
  P.tau = p->tau;
  P.omega = 1.0 / p->tau;
  P.guo = 1.0 - 0.5 / p->tau;
  P.four_pi_lb = 4.0 * M_PI * p->bjerrum;
  P.eps = 1.0 / (4.0 * M_PI * p->bjerrum);
  P.inv_2a0 = 1.0 / (2.0 * A0);
  P.selfmask = 0;
  for (int i = 1; i < lbe::kQ; ++i) {
    const bool self = (lbe::cx_of(i) == 0 || p->nx == 1) && (lbe::cy_of(i) == 0 || p->ny == 1) &&
                      (lbe::cz_of(i) == 0 || p->nz == 1);
    if (self) P.selfmask |= 1u << (i - 1);
  }
  if (p->boundary_rule == LBE_RULE_NODE) P.selfmask |= lbe::kPlainLaplacian;
  P.solid_factor = p->boundary_rule == LBE_RULE_NODE ? 1.0 : 2.0;
  // FP32 form
  lbe::P32 &Q = h->p32;
  memset(&Q, 0, sizeof(Q));
  Q.ns = p->nspecies;
  for (int k = 0; k < p->nspecies; ++k) {
    Q.zi[k] = (int)p->z[k];
    Q.zf[k] = (float)p->z[k];
    Q.rbd[k] = p->rho_bulk[k];
    Q.sd[k] = ldexp(p->rho_bulk[k], -lbe::kFixBits);
    Q.rb[k] = (float)Q.rbd[k];
    Q.s[k] = (float)Q.sd[k];
    Q.kq1[k] = (float)(-P.d[k] / 2.0 / Q.sd[k]);
    Q.kq2[k] = (float)(-P.d[k] / (2.0 * sqrt(2.0)) / Q.sd[k]);
  }
  for (int i = 0; i < lbe::kQ; ++i) {
    const int io = lbe::opp_of(i);
    // one rounding, mirrored for the opposite link so that ec[opp] = -ec
    Q.ec[i] = i <= 9 ? (float)P.e_dot_c[i] : -(float)P.e_dot_c[io];
  }
  Q.salt11 = p->nspecies == 2 && p->z[0] == 1.0 && p->z[1] == -1.0 && p->rho_bulk[0] == p->rho_bulk[1];
  Q.omega = (float)P.omega;
  Q.guo = (float)P.guo;
  Q.inv_2a0 = (float)P.inv_2a0;
}
}  // namespace lbe

extern "C" {

void lbe_default_params(lbe_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 1;
  p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
  p->tau = 1.0;
  p->bjerrum = 1.0;
  p->nspecies = 2;
  p->z[0] = 1.0;
  p->z[1] = -1.0;
  p->D[0] = p->D[1] = 0.05;
  p->rho_bulk[0] = p->rho_bulk[1] = 0.01;
  p->flow = 1;
  p->precision = LBE_FP64;
  p->poisson_tol = 1e-13;
  p->poisson_max_iter = 100000;
}

const char *lbe_last_error(const lbe_handle *h) {
  if (h) return h->err.c_str();
  return g_thread_err.empty() ? g_static_err : g_thread_err.c_str();
}

int lbe_create(const lbe_params *p, void *cuda_stream, lbe_handle **out) {
  if (!p || !out) return LBE_ERR_ARG;
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBE_ERR_ARG;
  if (p->nspecies < 1 || p->nspecies > LBE_MAX_SPECIES) return LBE_ERR_ARG;
  if (!(p->tau > 0.5) || !(p->bjerrum > 0.0)) return LBE_ERR_ARG;
  if (p->precision != LBE_FP64 && p->precision != LBE_FP32) return LBE_ERR_ARG;
  if (!(p->poisson_tol > 0.0) || p->poisson_max_iter < 1) return LBE_ERR_ARG;
  if (p->boundary_rule != LBE_RULE_MIDPLANE && p->boundary_rule != LBE_RULE_NODE) return LBE_ERR_ARG;
  // the FP32 form's multigrid and float-float stencils build in the doubling
  if (p->boundary_rule == LBE_RULE_NODE && p->precision != LBE_FP64) return LBE_ERR_ARG;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N >= (1LL << 31)) return LBE_ERR_ARG;  // 32-bit node indices in the kernels
  // FP32 kernels offset solute and velocity components in 32 bits
  if (p->precision == LBE_FP32 && N * (p->nspecies > 3 ? p->nspecies : 3) >= (1LL << 31)) return LBE_ERR_ARG;
  for (int k = 0; k < p->nspecies; ++k) {
    if (!(p->D[k] >= 0.0) || !(p->rho_bulk[k] >= 0.0)) return LBE_ERR_ARG;
    if (fabs(p->z[k]) > 4.0 || p->z[k] != floor(p->z[k])) return LBE_ERR_ARG;
    // the fixed-point unit of the FP32 form is relative to the bulk value
    if (p->precision == LBE_FP32 && !(p->rho_bulk[k] > 0.0)) return LBE_ERR_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->e_app[a])) return LBE_ERR_ARG;

  lbe_handle *h = new lbe_handle();
  h->prm = *p;
  h->geo = Geo{p->nx, p->ny, p->nz, p->periodic[0] != 0, p->periodic[1] != 0, p->periodic[2] != 0, N};
  lbe::fill_constants(h);

  const bool own = cuda_stream == nullptr;
  if (own) {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return LBE_ERR_CUDA;
    }
  } else {
    h->stream = (cudaStream_t)cuda_stream;
  }
  h->owns_stream = own;

  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  const size_t nd = sizeof(double) * (size_t)N, nf = sizeof(float) * (size_t)N;
  alloc((void **)&h->id, (size_t)N);
  alloc((void **)&h->mask, sizeof(uint32_t) * (size_t)N);
  alloc((void **)&h->phi, nd);
  alloc((void **)&h->psi_dev, sizeof(double) * (LBE_MAX_ELECTRODES + 1));
  if (fp32(h)) {
    alloc((void **)&h->f32[0], nf * lbe::kQ);  // one buffer: the populations are updated in place
    alloc((void **)&h->q, sizeof(int64_t) * (size_t)N * p->nspecies);
    alloc((void **)&h->qstar, sizeof(int64_t) * (size_t)N * p->nspecies);
    alloc((void **)&h->phifx, sizeof(int64_t) * (size_t)N);
    alloc((void **)&h->phi32, nf);
    alloc((void **)&h->u32, sizeof(float4) * (size_t)N);
    alloc((void **)&h->flag, sizeof(int));
    if (h->p32.salt11) alloc((void **)&h->lf, sizeof(float4) * (size_t)N);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->u32, 0, sizeof(float4) * (size_t)N, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
  } else {
    alloc((void **)&h->f[0], nd * lbe::kQ);
    if (p->flow) alloc((void **)&h->f[1], nd * lbe::kQ);
    alloc((void **)&h->n, nd * p->nspecies);
    alloc((void **)&h->nstar, nd * p->nspecies);
    alloc((void **)&h->u, nd * 3);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->u, 0, nd * 3, h->stream);
  }
  if (e == cudaSuccess) e = lbe::poisson_alloc(h);
  long long blocks = (N + lbe::kBlock - 1) / lbe::kBlock;
  h->qblk = (int)(blocks < 608 ? blocks : 608);
  alloc((void **)&h->qpart, sizeof(double) * h->qblk * LBE_MAX_ELECTRODES);
  alloc((void **)&h->qout, sizeof(double) * LBE_MAX_ELECTRODES);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->qhost, sizeof(double) * LBE_MAX_ELECTRODES);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    free_all(h);
    if (own) cudaStreamDestroy(h->stream);
    delete h;
    return LBE_ERR_CUDA;
  }
  *out = h;
  return LBE_OK;
}

int lbe_destroy(lbe_handle *h) {
  if (!h) return LBE_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  if (h->owns_stream) cudaStreamDestroy(h->stream);
  delete h;
  return LBE_OK;
}

int lbe_set_geometry(lbe_handle *h, const uint8_t *node_id, int n_electrodes, int on_device) {
  if (!h) return LBE_ERR_ARG;
  h->gen += 1;
  if (!node_id || n_electrodes < 0 || n_electrodes > LBE_MAX_ELECTRODES)
    return fail(h, LBE_ERR_ARG, "set_geometry: bad arguments");
  StreamGuard sg{h, h->owns_stream};
  const Geo &g = h->geo;
  std::vector<uint8_t> ids((size_t)g.N);
  if (on_device) {
    LBE_CK(h, cudaMemcpyAsync(ids.data(), node_id, (size_t)g.N, cudaMemcpyDeviceToHost, h->stream));
    LBE_CK(h, cudaStreamSynchronize(h->stream));
  } else {
    memcpy(ids.data(), node_id, (size_t)g.N);
  }
  // validate: ids in range; fluid nodes keep all 26 neighbours inside the box
  for (long long r = 0; r < g.N; ++r) {
    if (ids[r] > n_electrodes) return fail(h, LBE_ERR_GEOMETRY, "set_geometry: node id exceeds n_electrodes");
    if (ids[r]) continue;
    int x, y, z;
    lbe::coords(g, r, x, y, z);
    if ((!g.px && (x == 0 || x == g.nx - 1)) || (!g.py && (y == 0 || y == g.ny - 1)) ||
        (!g.pz && (z == 0 || z == g.nz - 1)))
      return fail(h, LBE_ERR_GEOMETRY, "set_geometry: fluid node on a non-periodic face");
  }
  LBE_CK(h, cudaMemcpyAsync(h->id, ids.data(), (size_t)g.N, cudaMemcpyHostToDevice, h->stream));
  LBE_CK(h, lbe::launch_build_mask(g, h->id, h->mask, h->stream));
  if (fp32(h)) LBE_CK(h, lbe::mg_setup(h));  // multigrid preconditioner of the FP32 Poisson solve
  lbe::poisson_drop_graphs(h);               // graphs capture the hierarchy
  LBE_CK(h, cudaStreamSynchronize(h->stream));  // ids is a host vector
  h->n_elec = n_electrodes;
  h->have_geometry = true;
  h->initialised = false;
  return LBE_OK;
}

// enqueue one Poisson solve and wait for its status (init, set_voltage)
static int solve_now(lbe_handle *h) {
  LBE_CK(h, lbe::poisson_reset_stats(h));
  int rc = lbe::poisson_enqueue(h, false);
  if (rc != LBE_OK) return rc;
  return lbe::poisson_status(h, &h->stats, nullptr);
}

int lbe_set_voltage(lbe_handle *h, const double *psi) {
  if (!h) return LBE_ERR_ARG;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "set_voltage: no geometry");
  if (!psi && h->n_elec > 0) return fail(h, LBE_ERR_ARG, "set_voltage: NULL psi");
  StreamGuard sg{h, h->owns_stream};
  for (int e = 0; e < h->n_elec; ++e) {
    if (!isfinite(psi[e])) return fail(h, LBE_ERR_ARG, "set_voltage: non-finite potential");
    if (fp32(h) && !(fabs(psi[e]) < lbe::kPhiMax))
      return fail(h, LBE_ERR_ARG, "set_voltage: the FP32 form holds potentials below 100 in magnitude");
  }
  bool same = h->initialised;
  for (int e = 0; e < h->n_elec; ++e) {
    same = same && h->psi[e] == psi[e];
    h->psi[e] = psi[e];
  }
  if (same) {
    // the electrodes already hold these potentials: upload them (the solid
    // nodes are rewritten with the same values) and keep the consistent state
    LBE_CK(h, lbe::launch_set_solid_phi(h));
    return LBE_OK;
  }
  h->gen += 1;
  if (!h->initialised) return LBE_OK;
  h->stats = lbe_stats{};
  // the FP32 form: the FP64 copy brought up to date, the electrodes set in
  // it, the whole of it back to fixed point
  LBE_CK(h, lbe::sync_phi64(h));
  LBE_CK(h, lbe::launch_set_solid_phi(h));
  if (fp32(h)) LBE_CK(h, lbe::launch_phi_from64(h));
  return solve_now(h);
}

int lbe_init(lbe_handle *h) {
  if (!h) return LBE_ERR_ARG;
  h->gen += 1;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "init: no geometry");
  StreamGuard sg{h, h->owns_stream};
  h->stats = lbe_stats{};
  h->cur = 0;
  if (fp32(h)) {
    LBE_CK(h, lbe::launch_init32(h));
    LBE_CK(h, lbe::launch_init_phi(h));
    LBE_CK(h, lbe::launch_phi_from64(h));
  } else {
    LBE_CK(h, lbe::launch_init_state(h));
  }
  int rc = solve_now(h);
  if (rc == LBE_OK) h->initialised = true;
  return rc;
}

// the FP32 form's range flag: copy_flag enqueues its read-back, flag_result
// evaluates it once the stream has been synchronised
static int copy_flag(lbe_handle *h) {
  if (!fp32(h)) return LBE_OK;
  LBE_CK(h, cudaMemcpyAsync(h->qhost, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  return LBE_OK;
}
static int flag_result(lbe_handle *h) {
  if (!fp32(h)) return LBE_OK;
  int flag = 0;
  memcpy(&flag, h->qhost, sizeof(int));
  if (flag)
    return fail(h, LBE_ERR_NONFINITE,
                "state out of range: fixed-point solute (|link flux| or |n| too large), potential (|phi| >= 100), "
                "solvent density or a NaN");
  return LBE_OK;
}
static int check_flags(lbe_handle *h) {
  if (!fp32(h)) return LBE_OK;
  const int rc = copy_flag(h);
  if (rc != LBE_OK) return rc;
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  return flag_result(h);
}

int lbe_step(lbe_handle *h, int nsteps) {
  if (!h) return LBE_ERR_ARG;
  h->gen += 1;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "step: call lbe_init first");
  if (nsteps < 0) return fail(h, LBE_ERR_ARG, "step: negative step count");
  StreamGuard sg{h, h->owns_stream};
  h->stats = lbe_stats{};
  const bool f32 = fp32(h);
  LBE_CK(h, lbe::poisson_reset_stats(h));
  for (int s = 0; s < nsteps; ++s) {
    LBE_CK(h, mark(h));
    LBE_CK(h, f32 ? lbe::launch_sweep32(h) : lbe::launch_sweep(h));
    LBE_CK(h, mark(h));
    h->launches += 1;
    // the FP32 form's advection also applies the next solve's warm start
    const bool fused_extrapolation = f32 && h->prm.flow;
    if (h->prm.flow) {
      LBE_CK(h, f32 ? lbe::launch_advect32(h, true) : lbe::launch_advect(h));
      h->launches += 1;
    } else if (f32) {
      int64_t *t = h->q;
      h->q = h->qstar;
      h->qstar = t;
    } else {
      double *t = h->n;
      h->n = h->nstar;
      h->nstar = t;
    }
    LBE_CK(h, mark(h));
    int rc = lbe::poisson_enqueue(h, true, fused_extrapolation);
    LBE_CK(h, mark(h));
    if (rc != LBE_OK) return rc;
    // a long call reads the solves' status now and then, so that a failed
    // solve ends it instead of every later step repeating the failure
    if ((s + 1) % 1024 == 0 && s + 1 < nsteps) {
      rc = lbe::poisson_status(h, nullptr, nullptr);
      if (rc != LBE_OK) return rc;
    }
  }
  // the solves ran without host synchronisation; their status and counts
  // are read once here, with the range flag, under one synchronisation (a
  // failed solve is reported at the end of the call)
  const int frc = copy_flag(h);
  if (frc != LBE_OK) return frc;
  long long graph_kernels = 0;
  int rc = lbe::poisson_status(h, &h->stats, &graph_kernels);
  h->launches += graph_kernels;
  if (h->profiling) {
    h->prof_iters += h->stats.poisson_iters;
    h->prof_solves += h->stats.poisson_solves;
    h->prof_steps += nsteps;
  }
  // a state out of range (range flag) explains a solve that failed after it
  const int frc2 = flag_result(h);
  return frc2 != LBE_OK ? frc2 : rc;
}

int lbe_induced_charge(lbe_handle *h, double *q_out, int out_on_device) {
  if (!h) return LBE_ERR_ARG;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "induced_charge: call lbe_init first");
  if (!q_out) return fail(h, LBE_ERR_ARG, "induced_charge: NULL output");
  StreamGuard sg{h, h->owns_stream};
  if (h->n_elec == 0) return LBE_OK;
  LBE_CK(h, lbe::sync_phi64(h));
  LBE_CK(h, lbe::launch_charge(h));
  const size_t bytes = sizeof(double) * h->n_elec;
  if (out_on_device) {
    LBE_CK(h, cudaMemcpyAsync(q_out, h->qout, bytes, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    LBE_CK(h, cudaMemcpyAsync(h->qhost, h->qout, bytes, cudaMemcpyDeviceToHost, h->stream));
    LBE_CK(h, cudaStreamSynchronize(h->stream));
    memcpy(q_out, h->qhost, bytes);
  }
  return LBE_OK;
}

int lbe_fields(lbe_handle *h, int which, void *out, int out_on_device) {
  if (!h) return LBE_ERR_ARG;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "fields: call lbe_init first");
  if (!out) return fail(h, LBE_ERR_ARG, "fields: NULL output");
  StreamGuard sg{h, h->owns_stream};
  const long long N = h->geo.N;
  size_t count;
  switch (which) {
    case LBE_FIELD_PHI: count = (size_t)N; break;
    case LBE_FIELD_N: count = (size_t)N * h->prm.nspecies; break;
    case LBE_FIELD_RHO: count = (size_t)N; break;
    case LBE_FIELD_U: count = (size_t)N * 3; break;
    case LBE_FIELD_F: count = (size_t)N * lbe::kQ; break;
    case LBE_FIELD_QNODE: count = (size_t)N; break;
    default: return fail(h, LBE_ERR_ARG, "fields: unknown field");
  }
  const size_t bytes = count * sizeof(double);
  double *dst = (double *)out;
  double *tmp = nullptr;
  if (!out_on_device) {
    LBE_CK(h, cudaMalloc(&tmp, bytes));
    dst = tmp;
  }
  cudaError_t e = lbe::sync_phi64(h);  // the potential and the node charges read the FP64 copy
  const bool f32 = fp32(h);
  if (e == cudaSuccess) switch (which) {
    case LBE_FIELD_PHI: e = cudaMemcpyAsync(dst, h->phi, bytes, cudaMemcpyDeviceToDevice, h->stream); break;
    case LBE_FIELD_N:
      e = f32 ? lbe::launch_n_to_double(h, dst)
              : cudaMemcpyAsync(dst, h->n, bytes, cudaMemcpyDeviceToDevice, h->stream);
      break;
    case LBE_FIELD_RHO:
      e = f32 ? lbe::launch_moments32(h, dst, nullptr, nullptr) : lbe::launch_moments(h, dst, nullptr);
      break;
    case LBE_FIELD_U:
      e = f32 ? lbe::launch_moments32(h, nullptr, dst, nullptr) : lbe::launch_moments(h, nullptr, dst);
      break;
    case LBE_FIELD_F:
      e = f32 ? lbe::launch_moments32(h, nullptr, nullptr, dst) : lbe::launch_gather_f(h, dst);
      break;
    case LBE_FIELD_QNODE: e = lbe::launch_charge_node(h, dst); break;
  }
  if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !out_on_device) e = cudaStreamSynchronize(h->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(h, LBE_ERR_CUDA, std::string("fields: ") + cudaGetErrorString(e));
  return LBE_OK;
}

int lbe_set_state(lbe_handle *h, const double *n, const double *phi, int on_device) {
  if (!h) return LBE_ERR_ARG;
  h->gen += 1;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "set_state: call lbe_init first");
  StreamGuard sg{h, h->owns_stream};
  const long long N = h->geo.N;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t nbytes = sizeof(double) * N * h->prm.nspecies;
  if (n && !fp32(h)) LBE_CK(h, cudaMemcpyAsync(h->n, n, nbytes, kind, h->stream));
  if (n && fp32(h)) {
    const double *src = n;
    double *tmp = nullptr;
    if (!on_device) {
      LBE_CK(h, cudaMalloc(&tmp, nbytes));
      LBE_CK(h, cudaMemcpyAsync(tmp, n, nbytes, cudaMemcpyHostToDevice, h->stream));
      src = tmp;
    }
    cudaError_t e = lbe::launch_n_from_double(h, src);
    if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    LBE_CK(h, e);
  }
  h->pw.history = 0;  // no warm-start extrapolation across a state change
  if (phi) {
    LBE_CK(h, cudaMemcpyAsync(h->phi, phi, sizeof(double) * N, kind, h->stream));
    LBE_CK(h, lbe::launch_set_solid_phi(h));
    if (fp32(h)) LBE_CK(h, lbe::launch_phi_from64(h));
  }
  if (!on_device) LBE_CK(h, cudaStreamSynchronize(h->stream));
  return check_flags(h);
}

// blob: header | populations (19N) | solute (ns N) | phi (N) | velocity (3N
// doubles, or N float4 records in the FP32 form) | phi of the previous kHist
// steps (kHist N, warm start of the next solve; header.history of them
// valid); every array in the form's own type (the FP32 form's potentials
// in its 64-bit fixed point), so that a restart is exact
struct BlobHeader {
  uint64_t magic;
  int64_t N;
  int32_t ns, flow, precision, history;
  int32_t aa_odd, pad;  // FP32 form: the kind of the next in-place step
};
static const uint64_t kMagic = 0x4c42457374763430ULL + lbe::kHist;  // format 4, history length

static void blob_sizes(const lbe_handle *h, size_t *fb, size_t *nb, size_t *pb, size_t *ub) {
  const size_t N = (size_t)h->geo.N;
  const bool f32 = h->prm.precision == LBE_FP32;
  *fb = N * lbe::kQ * (f32 ? sizeof(float) : sizeof(double));
  *nb = N * h->prm.nspecies * (f32 ? sizeof(int64_t) : sizeof(double));
  *pb = N * sizeof(double);
  *ub = N * (f32 ? sizeof(float4) : 3 * sizeof(double)) + lbe::kHist * N * sizeof(double);
}

int lbe_save_state(lbe_handle *h, void *blob, size_t *size) {
  if (!h || !size) return LBE_ERR_ARG;
  size_t fb, nb, pb, ub;
  blob_sizes(h, &fb, &nb, &pb, &ub);
  const size_t need = sizeof(BlobHeader) + fb + nb + pb + ub;
  if (!blob) {
    *size = need;
    return LBE_OK;
  }
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "save_state: call lbe_init first");
  if (*size < need) return fail(h, LBE_ERR_ARG, "save_state: blob too small");
  StreamGuard sg{h, h->owns_stream};
  const bool f32 = fp32(h);
  BlobHeader hd{kMagic, h->geo.N, h->prm.nspecies, h->prm.flow, h->prm.precision, h->pw.history, h->aa_odd ? 1 : 0,
                0};
  char *p = (char *)blob;
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  LBE_CK(h, cudaMemcpyAsync(p, f32 ? (void *)h->f32[0] : (void *)h->f[h->cur], fb, cudaMemcpyDeviceToHost,
                            h->stream));
  p += fb;
  LBE_CK(h, cudaMemcpyAsync(p, f32 ? (void *)h->q : (void *)h->n, nb, cudaMemcpyDeviceToHost, h->stream));
  p += nb;
  LBE_CK(h, cudaMemcpyAsync(p, f32 ? (void *)h->phifx : (void *)h->phi, pb, cudaMemcpyDeviceToHost, h->stream));
  p += pb;
  const size_t vb = ub - lbe::kHist * (size_t)h->geo.N * sizeof(double);
  LBE_CK(h, cudaMemcpyAsync(p, f32 ? (void *)h->u32 : (void *)h->u, vb, cudaMemcpyDeviceToHost, h->stream));
  p += vb;
  LBE_CK(h, cudaMemcpyAsync(p, h->pw.phi_prev, lbe::kHist * (size_t)h->geo.N * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  *size = need;
  return LBE_OK;
}

int lbe_load_state(lbe_handle *h, const void *blob, size_t size) {
  if (h) h->gen += 1;
  if (!h || !blob) return LBE_ERR_ARG;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "load_state: no geometry");
  size_t fb, nb, pb, ub;
  blob_sizes(h, &fb, &nb, &pb, &ub);
  const size_t need = sizeof(BlobHeader) + fb + nb + pb + ub;
  BlobHeader hd;
  if (size < need) return fail(h, LBE_ERR_ARG, "load_state: blob too small");
  memcpy(&hd, blob, sizeof(hd));
  if (hd.magic != kMagic || hd.N != h->geo.N || hd.ns != h->prm.nspecies || hd.flow != h->prm.flow ||
      hd.precision != h->prm.precision)
    return fail(h, LBE_ERR_ARG, "load_state: blob does not match this lattice");
  StreamGuard sg{h, h->owns_stream};
  const bool f32 = fp32(h);
  const char *p = (const char *)blob + sizeof(hd);
  h->cur = 0;
  h->aa_odd = hd.aa_odd != 0;
  h->pw.history = 0;
  LBE_CK(h, cudaMemcpyAsync(f32 ? (void *)h->f32[0] : (void *)h->f[0], p, fb, cudaMemcpyHostToDevice, h->stream));
  p += fb;
  LBE_CK(h, cudaMemcpyAsync(f32 ? (void *)h->q : (void *)h->n, p, nb, cudaMemcpyHostToDevice, h->stream));
  p += nb;
  LBE_CK(h, cudaMemcpyAsync(f32 ? (void *)h->phifx : (void *)h->phi, p, pb, cudaMemcpyHostToDevice, h->stream));
  p += pb;
  const size_t vb = ub - lbe::kHist * (size_t)h->geo.N * sizeof(double);
  LBE_CK(h, cudaMemcpyAsync(f32 ? (void *)h->u32 : (void *)h->u, p, vb, cudaMemcpyHostToDevice, h->stream));
  p += vb;
  LBE_CK(h, cudaMemcpyAsync(h->pw.phi_prev, p, lbe::kHist * (size_t)h->geo.N * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream));
  h->pw.history = hd.history < 0 ? 0 : (hd.history > lbe::kHist ? lbe::kHist : hd.history);
  if (f32) LBE_CK(h, lbe::launch_phi32_from_fx(h));
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  h->initialised = true;
  return LBE_OK;
}

int lbe_get_stats(const lbe_handle *h, lbe_stats *out) {
  if (!h || !out) return LBE_ERR_ARG;
  *out = h->stats;
  return LBE_OK;
}

int lbe_profile_begin(lbe_handle *h) {
  if (!h) return LBE_ERR_ARG;
  h->profiling = true;
  h->ev_used = 0;
  h->launches = 0;
  h->prof_iters = h->prof_solves = h->prof_steps = 0;
  return LBE_OK;
}

int lbe_profile_end(lbe_handle *h, lbe_profile *out) {
  if (!h || !out) return LBE_ERR_ARG;
  memset(out, 0, sizeof(*out));
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  const size_t steps = h->ev_used / 4;
  for (size_t s = 0; s < steps; ++s) {
    float a = 0.f, b = 0.f, c = 0.f;
    cudaEvent_t *e = &h->ev_pool[4 * s];
    LBE_CK(h, cudaEventElapsedTime(&a, e[0], e[1]));
    LBE_CK(h, cudaEventElapsedTime(&b, e[1], e[2]));
    LBE_CK(h, cudaEventElapsedTime(&c, e[2], e[3]));
    out->sweep_ms += a;
    out->advect_ms += b;
    out->poisson_ms += c;
  }
  out->sweep_launches = (long long)steps;
  out->advect_launches = h->prm.flow ? (long long)steps : 0;
  out->poisson_solves = h->prof_solves;
  out->poisson_iters = h->prof_iters;
  out->kernel_launches = h->launches;
  h->profiling = false;
  h->ev_used = 0;
  return LBE_OK;
}

}  // extern "C"
