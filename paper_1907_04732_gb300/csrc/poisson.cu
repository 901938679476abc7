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
// Reductions are deterministic: each block reduces in a fixed tree order and
// writes one partial; every consumer sums the partials in block order.
#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int kChunk = 16;        // iterations launched between host polls
constexpr int kRefresh = 50;      // true-residual refresh period

enum { P_PQ = 0, P_RZ0 = 1, P_RZ1 = 2, P_MAX = 3 };

__device__ __forceinline__ long long nb(const Geo &g, int x, int y, int z, int i) {
  return nbr(g, x, y, z, cx_of(i), cy_of(i), cz_of(i));
}

// diagonal of -lap_mod at a fluid node (links joining a node to itself, in
// boxes one node wide, cancel and are left out)
__device__ __forceinline__ double diag_of(uint32_t m, uint32_t selfmask) {
  double d = 0.0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const uint32_t b = 1u << (i - 1);
    if (selfmask & b) continue;
    d += (m & b) ? lapc_of(i) : 2.0 * lapc_of(i);
  }
  return d;
}

// lap_mod(v)(r) at a fluid node
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

// res = 4 pi l_B rho_el + lap_mod(phi); p = res/diag; partial rz, max
__global__ void __launch_bounds__(kBlock) k_cg_init(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                    const double *__restrict__ n, const double *__restrict__ phi,
                                                    double *__restrict__ rhs, double *__restrict__ res,
                                                    double *__restrict__ p, double *__restrict__ part, int nblk,
                                                    PoissonWork::Ctl *ctl) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->done = 0;
    ctl->iters = 0;
    ctl->status = 0;
  }
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

// convergence test after init or an update: reduce the max partials
__global__ void k_cg_check(const double *__restrict__ part, int nblk, PoissonWork::Ctl *ctl, double tol, int maxit,
                           int count_iteration) {
  if (ctl->done) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) v = fmax(v, part[P_MAX * nblk + b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) {
    if (count_iteration) ctl->iters += 1;
    ctl->res = v;
    if (v <= tol) {
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
__global__ void __launch_bounds__(kBlock) k_cg_matvec(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                      const double *__restrict__ p, double *__restrict__ q,
                                                      double *__restrict__ part, int nblk,
                                                      const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  double pq = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    int x, y, z;
    coords(g, r, x, y, z);
    const double p0 = p[r];
    double s = 0.0;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const uint32_t b = 1u << (i - 1);
      if ((P.selfmask & b) || !(m & b)) continue;
      s += lapc_of(i) * p[nb(g, x, y, z, i)];
    }
    const double qq = diag_of(m, P.selfmask) * p0 - s;
    q[r] = qq;
    pq += p0 * qq;
  }
  pq = block_reduce<false>(pq);
  if (threadIdx.x == 0) part[P_PQ * nblk + blockIdx.x] = pq;
}

// phi += alpha p, res -= alpha q; partial rz_new, max
__global__ void __launch_bounds__(kBlock) k_cg_update(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                      double *__restrict__ phi, double *__restrict__ res,
                                                      const double *__restrict__ p, const double *__restrict__ q,
                                                      double *__restrict__ part, int nblk,
                                                      const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  const int par = ctl->iters & 1;
  const double pq = sum_partials(part, nblk, P_PQ);
  const double rz = sum_partials(part, nblk, P_RZ0 + par);
  const double alpha = rz / pq;
  double rzn = 0.0, mx = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    phi[r] += alpha * p[r];
    const double rr = res[r] - alpha * q[r];
    res[r] = rr;
    const double d = diag_of(m, P.selfmask);
    rzn += rr * rr / d;
    mx = fmax(mx, fabs(rr) / d);
  }
  rzn = block_reduce<false>(rzn);
  if (threadIdx.x == 0) part[(P_RZ0 + (par ^ 1)) * nblk + blockIdx.x] = rzn;
  mx = block_reduce<true>(mx);
  if (threadIdx.x == 0) part[P_MAX * nblk + blockIdx.x] = mx;
}

// p = res/diag + beta p (ctl->iters already counts the finished iteration);
// every kRefresh iterations the recursive residual is replaced by the true one
__global__ void __launch_bounds__(kBlock) k_cg_direction(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                         const double *__restrict__ rhs, const double *__restrict__ phi,
                                                         double *__restrict__ res, double *__restrict__ p,
                                                         const double *__restrict__ part, int nblk,
                                                         const PoissonWork::Ctl *ctl) {
  if (ctl->done) return;
  const int it = ctl->iters;
  const int par = it & 1;
  const double rzn = sum_partials(part, nblk, P_RZ0 + par);
  const double rzo = sum_partials(part, nblk, P_RZ0 + (par ^ 1));
  const double beta = rzn / rzo;
  const bool refresh = (it % kRefresh) == 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[r];
    if (!(m & kFluidBit)) continue;
    const double d = diag_of(m, P.selfmask);
    p[r] = res[r] / d + beta * p[r];
    if (refresh) {
      int x, y, z;
      coords(g, r, x, y, z);
      res[r] = rhs[r] + lap_at(g, r, x, y, z, m, phi);
    }
  }
}

}  // namespace

cudaError_t poisson_alloc(lbe_handle *h) {
  PoissonWork &w = h->pw;
  const long long N = h->geo.N;
  long long blocks = (N + kBlock - 1) / kBlock;
  w.nblk = (int)(blocks < 608 ? blocks : 608);
  cudaError_t e;
  if ((e = cudaMalloc(&w.rhs, sizeof(double) * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.res, sizeof(double) * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.p, sizeof(double) * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.q, sizeof(double) * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.partial, sizeof(double) * 4 * w.nblk)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.ctl, sizeof(PoissonWork::Ctl))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&w.ctl_host, sizeof(PoissonWork::Ctl))) != cudaSuccess) return e;
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
  if (w.ctl_host) cudaFreeHost(w.ctl_host);
  w = PoissonWork{};
}

int poisson_solve(lbe_handle *h, int *iters, double *res) {
  PoissonWork &w = h->pw;
  const Geo &g = h->geo;
  const Phys &P = h->phys;
  cudaStream_t s = h->stream;
  const double tol = h->prm.poisson_tol;
  const int maxit = h->prm.poisson_max_iter;
  k_cg_init<<<w.nblk, kBlock, 0, s>>>(g, P, h->mask, h->n, h->phi, w.rhs, w.res, w.p, w.partial, w.nblk, w.ctl);
  k_cg_check<<<1, 32, 0, s>>>(w.partial, w.nblk, w.ctl, tol, maxit, 0);
  h->launches += 2;
  // the device counts iterations and stops at maxit; the host bound is a
  // second guard against a loop that never reports done
  const long long max_rounds = (long long)maxit / kChunk + 3;
  for (long long round = 0;; ++round) {
    if (round >= max_rounds) {
      h->err = "poisson: device never reported completion";
      return LBE_ERR_NOCONVERGE;
    }
    h->launches += 4 * kChunk;
    for (int c = 0; c < kChunk; ++c) {
      k_cg_matvec<<<w.nblk, kBlock, 0, s>>>(g, P, h->mask, w.p, w.q, w.partial, w.nblk, w.ctl);
      k_cg_update<<<w.nblk, kBlock, 0, s>>>(g, P, h->mask, h->phi, w.res, w.p, w.q, w.partial, w.nblk, w.ctl);
      k_cg_check<<<1, 32, 0, s>>>(w.partial, w.nblk, w.ctl, tol, maxit, 1);
      k_cg_direction<<<w.nblk, kBlock, 0, s>>>(g, P, h->mask, w.rhs, h->phi, w.res, w.p, w.partial, w.nblk,
                                               w.ctl);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.ctl_host, w.ctl, sizeof(PoissonWork::Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      h->err = std::string("poisson: ") + cudaGetErrorString(e);
      return LBE_ERR_CUDA;
    }
    if (w.ctl_host->done) break;
  }
  *iters = w.ctl_host->iters;
  *res = w.ctl_host->res;
  if (w.ctl_host->status == LBE_ERR_NOCONVERGE) {
    h->err = "poisson: no convergence within poisson_max_iter";
    return LBE_ERR_NOCONVERGE;
  }
  if (w.ctl_host->status == LBE_ERR_NONFINITE) {
    h->err = "poisson: non-finite residual";
    return LBE_ERR_NONFINITE;
  }
  return LBE_OK;
}

}  // namespace lbe
