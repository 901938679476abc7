// Poisson solve of the LBE step (Sec. "Imposing conducting boundary
// conditions"): find phi on fluid nodes such that
//     lap_mod(phi)(r) + 4 pi l_B rho_el(r) = 0,
// where lap_mod is Eq. DiscreteLaplacianModif (every fluid-solid link
// doubled) and solid nodes hold their electrode potential.  The paper relaxes
// with Eq. SOR and keeps the converged potential; this file reaches the same
// fixed point with Jacobi-preconditioned conjugate gradients on the symmetric
// positive definite fluid-node system, warm-started from the previous
// potential.  Stopping rule: max_r |res(r)|/diag(r) <= poisson_tol.
//
//  * FP64 form: CG in FP64 on phi itself.
//  * FP32 form: iterative refinement -- the residual is formed in FP64 from
//    the FP64 potential, the correction e (A e = res) is solved by CG in FP32
//    to a relative reduction, and phi += e in FP64; repeated until the FP64
//    residual meets the tolerance.
//
// Reductions are deterministic: each block reduces in a fixed tree order and
// writes one partial; every consumer sums the partials in block order.
#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int kChunk = 16;          // CG iterations launched between host polls
constexpr int kRefresh = 50;        // true-residual refresh period (FP64 form)
constexpr double kInnerEta = 2e-4;  // FP32 inner solve: relative reduction
constexpr int kMaxOuter = 40;       // FP32 form: refinement rounds per solve

enum { P_PQ = 0, P_RZ0 = 1, P_RZ1 = 2, P_MAX = 3 };

__device__ __forceinline__ long long nb(const Geo &g, int x, int y, int z, int i) {
  return nbr(g, x, y, z, cx_of(i), cy_of(i), cz_of(i));
}

// Link masks of the nearest (|c| = 1) and next-nearest neighbours.
__host__ __device__ constexpr uint32_t nn_bits() {
  uint32_t b = 0;
  for (int i = 1; i < kQ; ++i)
    if (c2_of(i) == 1) b |= 1u << (i - 1);
  return b;
}
constexpr uint32_t kNN = nn_bits();
constexpr uint32_t kNNN = ((1u << 18) - 1) & ~kNN;

// diagonal of -lap_mod at a fluid node: 1/3 per nearest and 1/6 per
// next-nearest link, doubled towards solid; links joining a node to itself
// (boxes one node wide) cancel and are left out.
__device__ __forceinline__ double diag_of(uint32_t m, uint32_t selfmask) {
  const uint32_t nself = ~selfmask;
  const int nn = __popc(kNN & nself), nns = __popc(kNN & nself & ~m);
  const int mm = __popc(kNNN & nself), mms = __popc(kNNN & nself & ~m);
  return (double)(2 * (nn + nns) + (mm + mms)) * (1.0 / 6.0);
}

// the same diagonal in the vector type of a CG kernel (no FP64 work in the
// FP32 kernels)
template <typename T>
__device__ __forceinline__ T diag_t(uint32_t m, uint32_t selfmask) {
  const uint32_t nself = ~selfmask;
  const int nn = __popc(kNN & nself), nns = __popc(kNN & nself & ~m);
  const int mm = __popc(kNNN & nself), mms = __popc(kNNN & nself & ~m);
  return (T)(2 * (nn + nns) + (mm + mms)) * (T)(1.0 / 6.0);
}

// lap_mod(v)(r) at a fluid node, FP64
__device__ __forceinline__ double lap_at(const Geo &g, long long r, int x, int y, int z, uint32_t m,
                                         const double *__restrict__ v) {
  const double v0 = v[r];
  double s = 0.0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const double vi = v[nb(g, x, y, z, i)];
    s += ((m & (1u << (i - 1))) ? lapc_of(i) : 2.0 * lapc_of(i)) * (vi - v0);
  }
  return s;
}

template <bool MAX>
__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double sh[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, t) : v + t;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double out = 0.0;
  if (threadIdx.x == 0) {
    out = sh[0];
    for (int w = 1; w < kBlock / 32; ++w) out = MAX ? fmax(out, sh[w]) : out + sh[w];
  }
  return out;  // valid in thread 0
}

// sum of the nblk partials of slot s, in block order; every thread gets it
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int nblk, int s) {
  __shared__ double sh_tot;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) v += part[(long long)s * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sh_tot = v;
  }
  __syncthreads();
  const double t = sh_tot;
  __syncthreads();
  return t;
}

__device__ __forceinline__ void reset_ctl(PoissonWork::Ctl *ctl) {
  if (ctl && blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->done = 0;
    ctl->iters = 0;
    ctl->status = 0;
  }
}

// FP64 form: res = 4 pi l_B rho_el + lap_mod(phi); p = res/diag
__global__ void __launch_bounds__(kBlock) k_cg_init64(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                      const double *__restrict__ n, const double *__restrict__ phi,
                                                      double *__restrict__ rhs, double *__restrict__ res,
                                                      double *__restrict__ p, double *__restrict__ part, int nblk,
                                                      PoissonWork::Ctl *ctl) {
  reset_ctl(ctl);
  double rz = 0.0, mx = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) {
      rhs[r] = 0.0;
      res[r] = 0.0;
      p[r] = 0.0;
      continue;
    }
    int x, y, z;
    coords(g, r, x, y, z);
    double q = 0.0;
    for (int k = 0; k < P.ns; ++k) q += P.z[k] * n[k * g.N + r];
    const double b = P.four_pi_lb * q;
    const double rr = b + lap_at(g, r, x, y, z, m, phi);
    const double d = diag_of(m, P.selfmask);
    rhs[r] = b;
    res[r] = rr;
    p[r] = rr / d;
    rz += rr * rr / d;
    mx = fmax(mx, fabs(rr) / d);
  }
  rz = block_reduce<false>(rz);
  if (threadIdx.x == 0) part[P_RZ0 * nblk + blockIdx.x] = rz;
  mx = block_reduce<true>(mx);
  if (threadIdx.x == 0) part[P_MAX * nblk + blockIdx.x] = mx;
}

// FP32 form, start of a refinement round: res64 = 4 pi l_B rho_el +
// lap_mod(phi64) in FP64 from the fixed-point solute amounts; its FP32 copy
// seeds the inner solve (e = 0, p = res/diag).  Partial max |res64|/diag.
__global__ void __launch_bounds__(kBlock) k_res64(const Geo g, const Phys P, const P32 P3,
                                                  const uint32_t *__restrict__ mask, const int64_t *__restrict__ qn,
                                                  const double *__restrict__ phi, float *__restrict__ res,
                                                  float *__restrict__ p, float *__restrict__ e,
                                                  double *__restrict__ part, int nblk, PoissonWork::Ctl *outer,
                                                  PoissonWork::Ctl *inner) {
  reset_ctl(outer);
  reset_ctl(inner);
  double rz = 0.0, mx = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) {
      res[r] = 0.f;
      p[r] = 0.f;
      e[r] = 0.f;
      continue;
    }
    int x, y, z;
    coords(g, r, x, y, z);
    double q = 0.0;
    for (int k = 0; k < P.ns; ++k) q += P.z[k] * (P3.rbd[k] + P3.sd[k] * (double)qn[k * g.N + r]);
    const double rr = P.four_pi_lb * q + lap_at(g, r, x, y, z, m, phi);
    const double d = diag_of(m, P.selfmask);
    const float rf = (float)rr, df = (float)d;
    res[r] = rf;
    p[r] = rf / df;
    e[r] = 0.f;
    rz += (double)(rf * (rf / df));
    mx = fmax(mx, fabs(rr) / d);
  }
  rz = block_reduce<false>(rz);
  if (threadIdx.x == 0) part[P_RZ0 * nblk + blockIdx.x] = rz;
  mx = block_reduce<true>(mx);
  if (threadIdx.x == 0) part[P_MAX * nblk + blockIdx.x] = mx;
}

// convergence test after an init or an update: reduce the max partials.
// tol_eff = max(tol, eta * first max), so eta > 0 asks for a relative
// reduction (FP32 inner solves).
__global__ void k_cg_check(const double *__restrict__ part, int nblk, PoissonWork::Ctl *ctl, double tol, double eta,
                           int maxit, int count_iteration) {
  if (ctl->done) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) v = fmax(v, part[P_MAX * nblk + b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) {
    if (count_iteration) ctl->iters += 1;
    else ctl->res0 = v;
    ctl->res = v;
    const double tol_eff = fmax(tol, eta * ctl->res0);
    if (v <= tol_eff) {
      ctl->done = 1;
    } else if (!(v == v) || v > 1e300) {
      ctl->done = 1;
      ctl->status = LBE_ERR_NONFINITE;
    } else if (ctl->iters >= maxit) {
      ctl->done = 1;
      ctl->status = LBE_ERR_NOCONVERGE;
    }
  }
}

// q = A p = -lap_mod(p) with p = 0 on solid nodes; partial p.q
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_matvec(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                                      const T *__restrict__ p, T *__restrict__ q,
                                                      double *__restrict__ part, int nblk,
                                                      const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  T pqt = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    int x, y, z;
    coords(g, r, x, y, z);
    const T p0 = p[r];
    T s = 0;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const uint32_t b = 1u << (i - 1);
      if ((selfmask & b) || !(m & b)) continue;
      s += (T)lapc_of(i) * p[nb(g, x, y, z, i)];
    }
    const T qq = diag_t<T>(m, selfmask) * p0 - s;
    q[r] = qq;
    pqt += p0 * qq;
  }
  double pq = block_reduce<false>((double)pqt);
  if (threadIdx.x == 0) part[P_PQ * nblk + blockIdx.x] = pq;
}

// x += alpha p, res -= alpha q; partial rz_new, max
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                                      T *__restrict__ xv, T *__restrict__ res,
                                                      const T *__restrict__ p, const T *__restrict__ q,
                                                      double *__restrict__ part, int nblk,
                                                      const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  const int par = ctl->iters & 1;
  const double pq = sum_partials(part, nblk, P_PQ);
  const double rz = sum_partials(part, nblk, P_RZ0 + par);
  const T alpha = (T)(rz / pq);
  T rzt = 0, mxt = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    xv[r] += alpha * p[r];
    const T rr = res[r] - alpha * q[r];
    res[r] = rr;
    const T dinv = (T)1 / diag_t<T>(m, selfmask);
    rzt += rr * rr * dinv;
    mxt = fmax(mxt, fabs(rr) * dinv);
  }
  double rzn = block_reduce<false>((double)rzt);
  double mx = (double)mxt;
  if (threadIdx.x == 0) part[(P_RZ0 + (par ^ 1)) * nblk + blockIdx.x] = rzn;
  mx = block_reduce<true>(mx);
  if (threadIdx.x == 0) part[P_MAX * nblk + blockIdx.x] = mx;
}

// p = res/diag + beta p (ctl->iters already counts the finished iteration);
// FP64 form: every kRefresh iterations the recursive residual is replaced by
// the true one
template <typename T, bool REFRESH>
__global__ void __launch_bounds__(kBlock) k_cg_direction(const Geo g, uint32_t selfmask,
                                                         const uint32_t *__restrict__ mask,
                                                         const double *__restrict__ rhs, const double *__restrict__ phi,
                                                         T *__restrict__ res, T *__restrict__ p,
                                                         const double *__restrict__ part, int nblk,
                                                         const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  const int it = ctl->iters;
  const int par = it & 1;
  const double rzn = sum_partials(part, nblk, P_RZ0 + par);
  const double rzo = sum_partials(part, nblk, P_RZ0 + (par ^ 1));
  const T beta = (T)(rzn / rzo);
  const bool refresh = REFRESH && (it % kRefresh) == 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    const T d = diag_t<T>(m, selfmask);
    p[r] = res[r] / d + beta * p[r];
    if (refresh) {
      int x, y, z;
      coords(g, r, x, y, z);
      res[r] = (T)(rhs[r] + lap_at(g, r, x, y, z, m, phi));
    }
  }
}

// FP32 form: phi64 += e on fluid nodes; refresh the FP32 copy everywhere
__global__ void k_correct(const Geo g, const uint32_t *__restrict__ mask, const float *__restrict__ e,
                          double *__restrict__ phi, float *__restrict__ phi32) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  double v = phi[r];
  if (e && (mask[r] & kFluidBit)) {
    v += (double)e[r];
    phi[r] = v;
  }
  phi32[r] = (float)v;
}

inline unsigned grid_for(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

// poll the control block of a solve (one D2H copy + stream sync)
int poll(lbe_handle *h, PoissonWork::Ctl *dev, PoissonWork::Ctl *host) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof(PoissonWork::Ctl), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("poisson: ") + cudaGetErrorString(e);
    return LBE_ERR_CUDA;
  }
  return LBE_OK;
}

int status_of(lbe_handle *h, const PoissonWork::Ctl &c) {
  if (c.status == LBE_ERR_NOCONVERGE) {
    h->err = "poisson: no convergence within poisson_max_iter";
    return LBE_ERR_NOCONVERGE;
  }
  if (c.status == LBE_ERR_NONFINITE) {
    h->err = "poisson: non-finite residual";
    return LBE_ERR_NONFINITE;
  }
  return LBE_OK;
}

// CG chunks until the control block says done (bounded by maxit on the
// device and by a round count on the host)
template <typename T, bool REFRESH>
int cg_loop(lbe_handle *h, T *x, T *res, T *p, T *q, const double *rhs, const double *phi, PoissonWork::Ctl *ctl,
            PoissonWork::Ctl *ctl_host, double tol, double eta, int maxit) {
  PoissonWork &w = h->pw;
  const Geo &g = h->geo;
  const uint32_t sm = h->phys.selfmask;
  cudaStream_t s = h->stream;
  const long long max_rounds = (long long)maxit / kChunk + 3;
  for (long long round = 0;; ++round) {
    if (round >= max_rounds) {
      h->err = "poisson: device never reported completion";
      return LBE_ERR_NOCONVERGE;
    }
    for (int c = 0; c < kChunk; ++c) {
      k_cg_matvec<T><<<w.nblk, kBlock, 0, s>>>(g, sm, h->mask, p, q, w.partial, w.nblk, ctl);
      k_cg_update<T><<<w.nblk, kBlock, 0, s>>>(g, sm, h->mask, x, res, p, q, w.partial, w.nblk, ctl);
      k_cg_check<<<1, 32, 0, s>>>(w.partial, w.nblk, ctl, tol, eta, maxit, 1);
      k_cg_direction<T, REFRESH><<<w.nblk, kBlock, 0, s>>>(g, sm, h->mask, rhs, phi, res, p, w.partial, w.nblk, ctl);
    }
    h->launches += 4 * kChunk;
    int rc = poll(h, ctl, ctl_host);
    if (rc != LBE_OK) return rc;
    if (ctl_host->done) return LBE_OK;
  }
}

}  // namespace

cudaError_t poisson_alloc(lbe_handle *h) {
  PoissonWork &w = h->pw;
  const long long N = h->geo.N;
  long long blocks = (N + kBlock - 1) / kBlock;
  w.nblk = (int)(blocks < 608 ? blocks : 608);
  cudaError_t e;
  if (h->prm.precision == LBE_FP64) {
    if ((e = cudaMalloc(&w.rhs, sizeof(double) * N)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.res, sizeof(double) * N)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.p, sizeof(double) * N)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.q, sizeof(double) * N)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMalloc(&h->pw32, sizeof(float) * 4 * N)) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&w.partial, sizeof(double) * 4 * w.nblk)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.ctl, 2 * sizeof(PoissonWork::Ctl))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&w.ctl_host, 2 * sizeof(PoissonWork::Ctl))) != cudaSuccess) return e;
  return cudaSuccess;
}

void poisson_free(lbe_handle *h) {
  PoissonWork &w = h->pw;
  cudaFree(w.rhs);
  cudaFree(w.res);
  cudaFree(w.p);
  cudaFree(w.q);
  cudaFree(w.partial);
  cudaFree(w.ctl);
  cudaFree(h->pw32);
  h->pw32 = nullptr;
  if (w.ctl_host) cudaFreeHost(w.ctl_host);
  w = PoissonWork{};
}

int poisson_solve(lbe_handle *h, int *iters, double *res) {
  PoissonWork &w = h->pw;
  const double tol = h->prm.poisson_tol;
  const int maxit = h->prm.poisson_max_iter;
  k_cg_init64<<<w.nblk, kBlock, 0, h->stream>>>(h->geo, h->phys, h->mask, h->n, h->phi, w.rhs, w.res, w.p,
                                                 w.partial, w.nblk, w.ctl);
  k_cg_check<<<1, 32, 0, h->stream>>>(w.partial, w.nblk, w.ctl, tol, 0.0, maxit, 0);
  h->launches += 2;
  int rc = cg_loop<double, true>(h, h->phi, w.res, w.p, w.q, w.rhs, h->phi, w.ctl, w.ctl_host, tol, 0.0, maxit);
  *iters = w.ctl_host->iters;
  *res = w.ctl_host->res;
  if (rc != LBE_OK) return rc;
  return status_of(h, *w.ctl_host);
}

int poisson_solve_mixed(lbe_handle *h, int *iters, double *res) {
  PoissonWork &w = h->pw;
  const Geo &g = h->geo;
  const long long N = g.N;
  float *r32 = h->pw32, *p32 = h->pw32 + N, *q32 = h->pw32 + 2 * N, *e32 = h->pw32 + 3 * N;
  PoissonWork::Ctl *outer = w.ctl + 1, *outer_h = w.ctl_host + 1;
  const double tol = h->prm.poisson_tol;
  const int maxit = h->prm.poisson_max_iter;
  int total = 0;
  *res = 0.0;
  for (int round = 0; round < kMaxOuter; ++round) {
    // FP64 residual of the current potential; seeds the inner FP32 solve and
    // resets both control blocks
    k_res64<<<w.nblk, kBlock, 0, h->stream>>>(g, h->phys, h->p32, h->mask, h->q, h->phi, r32, p32, e32, w.partial,
                                               w.nblk, outer, w.ctl);
    k_cg_check<<<1, 32, 0, h->stream>>>(w.partial, w.nblk, outer, tol, 0.0, 1 << 30, 0);
    // inner solve's starting residual (same partials), relative stop
    k_cg_check<<<1, 32, 0, h->stream>>>(w.partial, w.nblk, w.ctl, 0.0, kInnerEta, maxit, 0);
    h->launches += 3;
    int rc = poll(h, outer, outer_h);
    if (rc != LBE_OK) return rc;
    *res = outer_h->res;
    if (!(outer_h->res == outer_h->res) || outer_h->res > 1e300) {
      h->err = "poisson: non-finite residual";
      return LBE_ERR_NONFINITE;
    }
    if (outer_h->done) {
      *iters = total;
      return LBE_OK;
    }
    rc = cg_loop<float, false>(h, e32, r32, p32, q32, nullptr, nullptr, w.ctl, w.ctl_host, 0.0, kInnerEta,
                               maxit - total);
    total += w.ctl_host->iters;
    if (rc != LBE_OK) return rc;
    if (w.ctl_host->status == LBE_ERR_NONFINITE) return status_of(h, *w.ctl_host);
    k_correct<<<grid_for(N), kBlock, 0, h->stream>>>(g, h->mask, e32, h->phi, h->phi32);
    h->launches += 1;
    if (total >= maxit) {
      *iters = total;
      h->err = "poisson: no convergence within poisson_max_iter";
      return LBE_ERR_NOCONVERGE;
    }
  }
  *iters = total;
  h->err = "poisson: refinement did not reach the tolerance";
  return LBE_ERR_NOCONVERGE;
}

cudaError_t launch_phi32_sync(lbe_handle *h) {
  // phi32 = (float) phi64 everywhere (after init / set_state / set_voltage)
  k_correct<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->mask, nullptr, h->phi, h->phi32);
  return cudaGetLastError();
}

}  // namespace lbe
