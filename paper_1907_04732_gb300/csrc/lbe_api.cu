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

void free_all(lbe_handle *h) {
  cudaFree(h->id);
  cudaFree(h->mask);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->n);
  cudaFree(h->nstar);
  cudaFree(h->phi);
  cudaFree(h->u);
  cudaFree(h->qpart);
  cudaFree(h->qout);
  cudaFree(h->psi_dev);
  if (h->qhost) cudaFreeHost(h->qhost);
  lbe::poisson_free(h);
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

const char *lbe_last_error(const lbe_handle *h) { return h ? h->err.c_str() : g_static_err; }

int lbe_create(const lbe_params *p, void *cuda_stream, lbe_handle **out) {
  if (!p || !out) return LBE_ERR_ARG;
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBE_ERR_ARG;
  if (p->nspecies < 1 || p->nspecies > LBE_MAX_SPECIES) return LBE_ERR_ARG;
  if (!(p->tau > 0.5) || !(p->bjerrum > 0.0)) return LBE_ERR_ARG;
  if (p->precision != LBE_FP64 && p->precision != LBE_FP32) return LBE_ERR_ARG;
  if (!(p->poisson_tol > 0.0) || p->poisson_max_iter < 1) return LBE_ERR_ARG;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 40)) return LBE_ERR_ARG;
  for (int k = 0; k < p->nspecies; ++k) {
    if (!(p->D[k] >= 0.0) || !(p->rho_bulk[k] >= 0.0)) return LBE_ERR_ARG;
    if (fabs(p->z[k]) > 4.0 || p->z[k] != floor(p->z[k])) return LBE_ERR_ARG;
  }
  if (p->precision == LBE_FP32) return LBE_ERR_ARG;  // not built in this library version

  lbe_handle *h = new lbe_handle();
  h->prm = *p;
  h->geo = Geo{p->nx, p->ny, p->nz, p->periodic[0] != 0, p->periodic[1] != 0, p->periodic[2] != 0, N};
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

  bool own = cuda_stream == nullptr;
  if (own) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return LBE_ERR_CUDA;
    }
  } else {
    h->stream = (cudaStream_t)cuda_stream;
  }
  h->owns_stream = own;

  auto alloc = [&](void **ptr, size_t bytes) { return cudaMalloc(ptr, bytes); };
  cudaError_t e = cudaSuccess;
  const size_t nd = sizeof(double) * (size_t)N;
  if (e == cudaSuccess) e = alloc((void **)&h->id, (size_t)N);
  if (e == cudaSuccess) e = alloc((void **)&h->mask, sizeof(uint32_t) * (size_t)N);
  if (e == cudaSuccess) e = alloc((void **)&h->f[0], nd * lbe::kQ);
  if (e == cudaSuccess && p->flow) e = alloc((void **)&h->f[1], nd * lbe::kQ);
  if (e == cudaSuccess) e = alloc((void **)&h->n, nd * p->nspecies);
  if (e == cudaSuccess) e = alloc((void **)&h->nstar, nd * p->nspecies);
  if (e == cudaSuccess) e = alloc((void **)&h->phi, nd);
  if (e == cudaSuccess) e = alloc((void **)&h->u, nd * 3);
  if (e == cudaSuccess) e = alloc((void **)&h->psi_dev, sizeof(double) * (LBE_MAX_ELECTRODES + 1));
  if (e == cudaSuccess) e = lbe::poisson_alloc(h);
  if (e == cudaSuccess) {
    long long blocks = (N + lbe::kBlock - 1) / lbe::kBlock;
    h->qblk = (int)(blocks < 608 ? blocks : 608);
    e = alloc((void **)&h->qpart, sizeof(double) * h->qblk * LBE_MAX_ELECTRODES);
  }
  if (e == cudaSuccess) e = alloc((void **)&h->qout, sizeof(double) * LBE_MAX_ELECTRODES);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->qhost, sizeof(double) * LBE_MAX_ELECTRODES);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->u, 0, nd * 3, h->stream);
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
  LBE_CK(h, cudaStreamSynchronize(h->stream));  // ids is a host vector
  h->n_elec = n_electrodes;
  h->have_geometry = true;
  h->initialised = false;
  return LBE_OK;
}

static int solve(lbe_handle *h) {
  int it = 0;
  double res = 0.0;
  int rc = lbe::poisson_solve(h, &it, &res);
  h->stats.poisson_iters += it;
  h->stats.poisson_solves += 1;
  if (it > h->stats.poisson_max_iters) h->stats.poisson_max_iters = it;
  h->stats.poisson_residual = res;
  return rc;
}

int lbe_set_voltage(lbe_handle *h, const double *psi) {
  if (!h) return LBE_ERR_ARG;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "set_voltage: no geometry");
  if (!psi && h->n_elec > 0) return fail(h, LBE_ERR_ARG, "set_voltage: NULL psi");
  StreamGuard sg{h, h->owns_stream};
  for (int e = 0; e < h->n_elec; ++e) {
    if (!isfinite(psi[e])) return fail(h, LBE_ERR_ARG, "set_voltage: non-finite potential");
    h->psi[e] = psi[e];
  }
  if (!h->initialised) return LBE_OK;
  h->stats = lbe_stats{};
  LBE_CK(h, lbe::launch_set_solid_phi(h));
  return solve(h);
}

int lbe_init(lbe_handle *h) {
  if (!h) return LBE_ERR_ARG;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "init: no geometry");
  StreamGuard sg{h, h->owns_stream};
  h->stats = lbe_stats{};
  h->cur = 0;
  LBE_CK(h, lbe::launch_init_state(h));
  int rc = solve(h);
  if (rc == LBE_OK) h->initialised = true;
  return rc;
}

int lbe_step(lbe_handle *h, int nsteps) {
  if (!h) return LBE_ERR_ARG;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "step: call lbe_init first");
  if (nsteps < 0) return fail(h, LBE_ERR_ARG, "step: negative step count");
  StreamGuard sg{h, h->owns_stream};
  h->stats = lbe_stats{};
  for (int s = 0; s < nsteps; ++s) {
    LBE_CK(h, mark(h));
    LBE_CK(h, lbe::launch_sweep(h));
    LBE_CK(h, mark(h));
    h->launches += 1;
    if (h->prm.flow) {
      LBE_CK(h, lbe::launch_advect(h));
      h->launches += 1;
    } else {
      double *t = h->n;
      h->n = h->nstar;
      h->nstar = t;
    }
    LBE_CK(h, mark(h));
    const long long it0 = h->stats.poisson_iters;
    int rc = solve(h);
    LBE_CK(h, mark(h));
    if (h->profiling) {
      h->prof_iters += h->stats.poisson_iters - it0;
      h->prof_solves += 1;
      h->prof_steps += 1;
    }
    if (rc != LBE_OK) return rc;
  }
  return LBE_OK;
}

int lbe_induced_charge(lbe_handle *h, double *q_out, int out_on_device) {
  if (!h) return LBE_ERR_ARG;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "induced_charge: call lbe_init first");
  if (!q_out) return fail(h, LBE_ERR_ARG, "induced_charge: NULL output");
  StreamGuard sg{h, h->owns_stream};
  if (h->n_elec == 0) return LBE_OK;
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
    default: return fail(h, LBE_ERR_ARG, "fields: unknown field");
  }
  const size_t bytes = count * sizeof(double);
  double *dst = (double *)out;
  double *tmp = nullptr;
  if (!out_on_device) {
    LBE_CK(h, cudaMalloc(&tmp, bytes));
    dst = tmp;
  }
  cudaError_t e = cudaSuccess;
  switch (which) {
    case LBE_FIELD_PHI: e = cudaMemcpyAsync(dst, h->phi, bytes, cudaMemcpyDeviceToDevice, h->stream); break;
    case LBE_FIELD_N: e = cudaMemcpyAsync(dst, h->n, bytes, cudaMemcpyDeviceToDevice, h->stream); break;
    case LBE_FIELD_RHO: e = lbe::launch_moments(h, dst, nullptr); break;
    case LBE_FIELD_U: e = lbe::launch_moments(h, nullptr, dst); break;
    case LBE_FIELD_F: e = lbe::launch_gather_f(h, dst); break;
  }
  if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !out_on_device) e = cudaStreamSynchronize(h->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(h, LBE_ERR_CUDA, std::string("fields: ") + cudaGetErrorString(e));
  return LBE_OK;
}

int lbe_set_state(lbe_handle *h, const double *n, const double *phi, int on_device) {
  if (!h) return LBE_ERR_ARG;
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "set_state: call lbe_init first");
  StreamGuard sg{h, h->owns_stream};
  const long long N = h->geo.N;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n) LBE_CK(h, cudaMemcpyAsync(h->n, n, sizeof(double) * N * h->prm.nspecies, kind, h->stream));
  if (phi) {
    LBE_CK(h, cudaMemcpyAsync(h->phi, phi, sizeof(double) * N, kind, h->stream));
    LBE_CK(h, lbe::launch_set_solid_phi(h));
  }
  if (!on_device) LBE_CK(h, cudaStreamSynchronize(h->stream));
  return LBE_OK;
}

// blob: header | f[cur] (19N) | n (ns N) | phi (N) | u (3N)
struct BlobHeader {
  uint64_t magic;
  int64_t N;
  int32_t ns, flow;
};
static const uint64_t kMagic = 0x4c42453634763031ULL;  // "LBE64v01"

int lbe_save_state(lbe_handle *h, void *blob, size_t *size) {
  if (!h || !size) return LBE_ERR_ARG;
  const long long N = h->geo.N;
  const int ns = h->prm.nspecies;
  const size_t need = sizeof(BlobHeader) + sizeof(double) * (size_t)N * (lbe::kQ + ns + 1 + 3);
  if (!blob) {
    *size = need;
    return LBE_OK;
  }
  if (!h->initialised) return fail(h, LBE_ERR_STATE, "save_state: call lbe_init first");
  if (*size < need) return fail(h, LBE_ERR_ARG, "save_state: blob too small");
  StreamGuard sg{h, h->owns_stream};
  BlobHeader hd{kMagic, N, ns, h->prm.flow};
  char *p = (char *)blob;
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const size_t nd = sizeof(double) * (size_t)N;
  LBE_CK(h, cudaMemcpyAsync(p, h->f[h->cur], nd * lbe::kQ, cudaMemcpyDeviceToHost, h->stream));
  p += nd * lbe::kQ;
  LBE_CK(h, cudaMemcpyAsync(p, h->n, nd * ns, cudaMemcpyDeviceToHost, h->stream));
  p += nd * ns;
  LBE_CK(h, cudaMemcpyAsync(p, h->phi, nd, cudaMemcpyDeviceToHost, h->stream));
  p += nd;
  LBE_CK(h, cudaMemcpyAsync(p, h->u, nd * 3, cudaMemcpyDeviceToHost, h->stream));
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  *size = need;
  return LBE_OK;
}

int lbe_load_state(lbe_handle *h, const void *blob, size_t size) {
  if (!h || !blob) return LBE_ERR_ARG;
  if (!h->have_geometry) return fail(h, LBE_ERR_STATE, "load_state: no geometry");
  const long long N = h->geo.N;
  const int ns = h->prm.nspecies;
  const size_t need = sizeof(BlobHeader) + sizeof(double) * (size_t)N * (lbe::kQ + ns + 1 + 3);
  BlobHeader hd;
  if (size < need) return fail(h, LBE_ERR_ARG, "load_state: blob too small");
  memcpy(&hd, blob, sizeof(hd));
  if (hd.magic != kMagic || hd.N != N || hd.ns != ns || hd.flow != h->prm.flow)
    return fail(h, LBE_ERR_ARG, "load_state: blob does not match this lattice");
  StreamGuard sg{h, h->owns_stream};
  const char *p = (const char *)blob + sizeof(hd);
  const size_t nd = sizeof(double) * (size_t)N;
  h->cur = 0;
  LBE_CK(h, cudaMemcpyAsync(h->f[0], p, nd * lbe::kQ, cudaMemcpyHostToDevice, h->stream));
  p += nd * lbe::kQ;
  LBE_CK(h, cudaMemcpyAsync(h->n, p, nd * ns, cudaMemcpyHostToDevice, h->stream));
  p += nd * ns;
  LBE_CK(h, cudaMemcpyAsync(h->phi, p, nd, cudaMemcpyHostToDevice, h->stream));
  p += nd;
  LBE_CK(h, cudaMemcpyAsync(h->u, p, nd * 3, cudaMemcpyHostToDevice, h->stream));
  LBE_CK(h, cudaStreamSynchronize(h->stream));
  h->initialised = true;
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

int lbe_get_stats(const lbe_handle *h, lbe_stats *out) {
  if (!h || !out) return LBE_ERR_ARG;
  *out = h->stats;
  return LBE_OK;
}

}  // extern "C"
