// Reverse-mode derivative (adjoint) of the induced charge after T steps of
// the FP32 form with the solvent at rest (declarations in include/lbe.h).
//
// Forward (Sec. "Lattice Boltzmann Electrokinetics", flow off):
//   n^0 = rho_b (1 - chi),  phi^t = Poisson(n^t),
//   n^{t+1} = n^t - sum_i J_i(n^t, phi^t)     (Eq. LF2 link fluxes)
//   S = sum_e c_e Q_e(phi^T)                   (Eq. Qelec)
// The derivatives are those of the soft-occupancy reading of the method
// (row-scaled Poisson with a chi (psi - phi) term, link factor
// 1 + (chi - chi')^2, ion-link openness (1 - chi)(1 - chi'), chi-weighted
// charge), evaluated at the binary geometry of the handle, where that
// reading is the method itself.
//
// Backward, t = T .. 0:
//   phibar^T = dS/dphi^T                      (seed; direct chi terms of Q)
//   mu^t: A mu = -phibar on fluid nodes       (adjoint Poisson, the FP32
//         refinement solver with multigrid; A is symmetric), and on solid
//         nodes mu_s = sum 2 w mu_fluid - phibar_s
//   nbar^t += -4 pi l_B z_k mu;  psibar_e -= sum_{s in e} mu_s;  chibar += ...
//   t > 0: the flux step's transpose gives nbar^{t-1}, phibar^{t-1}, Dbar,
//          chibar (openness)
//   t = 0: rho_bbar += sum nbar^0, chibar -= rho_b sum_k nbar^0
// The forward states of a step are recomputed from checkpoints: either
// taken every K steps (two-level checkpointing: the states of one segment
// are kept while it is differentiated), or placed by the binomial schedule
// of Griewank and Walther ("revolve") within a device-memory budget, which
// reverses T steps with s checkpoint slots by recomputing each step at most
// r times, r the smallest with C(s + r, s) >= T.  Parameter sums are FP64,
// in a fixed order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fp32_device.cuh"

namespace lbe {

constexpr int kAdjSlots = LBE_MAX_ELECTRODES + LBE_MAX_SPECIES + 1;  // psibar, Dbar, rho_bbar
constexpr int kSlotD = LBE_MAX_ELECTRODES, kSlotRho = LBE_MAX_ELECTRODES + LBE_MAX_SPECIES;

struct AdjWork {
  long long N = 0;
  int T = 0, every = 0, nseg = 0, nblk = 0;
  long long gen = -1;  // handle generation after the forward pass
  bool ready = false;
  // binomial schedule: checkpoint slots (ck_* hold nseg + 1 of them then:
  // slot 0 the initial state, slots 1.. the forward pass's first descent,
  // slot nseg the final state); 0 = uniform checkpoints
  int revolve_slots = 0;
  int64_t *ck_q = nullptr;  // checkpoints [nseg + 1][2N] (the last: time T)
  double *ck_phi = nullptr;   // [nseg + 1][N] (the fixed-point potential's 8 bytes per node)
  double *ck_prev = nullptr;  // [nseg + 1][kHist N]: the warm start's history
  std::vector<char> ck_hist;
  int64_t *st_q = nullptr;  // states of one segment [every][2N]
  float *st_phi = nullptr;  // [every][N]
  float *lam = nullptr, *lam2 = nullptr;  // nbar [2][N]
  float *phibar = nullptr;
  double *mu = nullptr, *rhs = nullptr, *chibar = nullptr;
  double *mu_prev = nullptr;  // mu of the previous solve (warm start by extrapolation)
  float *mu_hi = nullptr, *mu_lo = nullptr;  // mu as two floats (float-float residual)
  int nsolved = 0;            // solves since the seed
  double *part = nullptr, *acc = nullptr;  // [kAdjSlots][nblk], [kAdjSlots]
  double q[LBE_MAX_ELECTRODES] = {};
  std::vector<cudaEvent_t> ev;  // phase timing: 2 + 2 per step of a segment
};

namespace {

struct Weights {
  double c[LBE_MAX_ELECTRODES + 1];  // index = electrode id (0 unused)
};

// node index r -> coordinates and the in-box neighbour along link l (-1
// outside a non-periodic face)
__device__ __forceinline__ long long link_nbr(const Geo &g, int x, int y, int z, int l) {
  return nbr(g, x, y, z, cx_of(l), cy_of(l), cz_of(l));
}

__device__ __forceinline__ float phi_at(long long j, const uint8_t *__restrict__ id, const float *__restrict__ phi,
                                        const Weights &psi) {
  const int e = id[j];
  return e ? (float)psi.c[e] : phi[j];
}

// block partial sums of the slots [S0, S1) in a fixed order
template <int S0, int S1>
__device__ __forceinline__ void block_partials(const double *v, double *__restrict__ part, int nblk) {
  __shared__ double sh[kBlock / 32][S1 - S0];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int k = 0; k < S1 - S0; ++k) {
    double a = v[k];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[wid][k] = a;
  }
  __syncthreads();
  if (t < S1 - S0) {
    double a = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) a += sh[w][t];
    part[(long long)(S0 + t) * nblk + blockIdx.x] = a;
  }
}

// coordinates of node r (32-bit arithmetic; lattices have < 2^31 nodes)
__device__ __forceinline__ void coords32(const Geo &g, int r, int &x, int &y, int &z) {
  x = r % g.nx;
  const int t = r / g.nx;
  y = t % g.ny;
  z = t / g.ny;
}

// seed of the backward pass: phibar = dS/dphi^T and the direct chi terms of
// S = sum_e c_e Q_e (links from electrode nodes to fluid, weight 2 w)
__global__ void __launch_bounds__(kBlock) k_adj_seed(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                     const uint8_t *__restrict__ id, const float *__restrict__ phi,
                                                     const Weights cq, const Weights psi, int soft,
                                                     float *__restrict__ phibar, double *__restrict__ chibar) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    coords32(g, (int)r, x, y, z);
    const uint32_t m = mask[r];
    const int e = id[r];
    const double pr = phi_at(r, id, phi, psi);
    double pb = 0.0, cb = 0.0;
    for (int l = 1; l < kQ; ++l) {
      const uint32_t b = 1u << (l - 1);
      if (P.selfmask & b) continue;
      const double w = lapc_of(l);
      const long long j = link_nbr(g, x, y, z, l);
      if (j < 0 || j == r) continue;
      const int ej = id[j];
      const double pj = phi_at(j, id, phi, psi);
      if (!e) {
        if (m & b) {
          cb += cq.c[soft] * (-P.eps) * w * (pj - pr);
        } else {
          pb += cq.c[ej] * (-P.eps) * 2.0 * w;
          cb += cq.c[ej] * 4.0 * P.eps * w * (pr - pj);
        }
      } else {
        if (m & b) {
          pb += cq.c[e] * P.eps * 2.0 * w;
          cb += cq.c[e] * (-4.0) * P.eps * w * (pj - pr);
        } else if (ej && ej != e) {
          cb += cq.c[ej] * P.eps * w * (pr - pj);
        }
      }
    }
    phibar[r] = (float)pb;
    chibar[r] += cb;
  }
}

// warm start of the adjoint solve: mu <- 2 mu(t+1) - mu(t+2) on fluid nodes
// (linear extrapolation in time; the solution does not depend on the start),
// remembering mu(t+1).  Unlike the forward potential, the quadratic start
// measured worse here: 25.5 k instead of 19.0 k adjoint CG iterations over
// 2000 steps of the porous electrode.
__global__ void k_adj_extrapolate(long long N, const uint32_t *__restrict__ mask, double *__restrict__ mu,
                                  double *__restrict__ prev, int have) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    if (!(mask[r] & kFluidBit)) continue;
    const double v = mu[r];
    if (have) mu[r] = 2.0 * v - prev[r];
    prev[r] = v;
  }
}

// right-hand side of the adjoint Poisson solve: -phibar on fluid nodes
__global__ void k_adj_rhs(long long N, const uint32_t *__restrict__ mask, const float *__restrict__ phibar,
                          double *__restrict__ rhs) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
    rhs[r] = (mask[r] & kFluidBit) ? -(double)phibar[r] : 0.0;
}

// after the adjoint solve: nbar += -4 pi l_B z mu (fluid), mu on solid nodes,
// psibar, and the chi terms of the Poisson equation
__global__ void __launch_bounds__(kBlock) k_adj_post(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                     const uint8_t *__restrict__ id, const float *__restrict__ phi,
                                                     const float *__restrict__ phibar, const double *__restrict__ mu,
                                                     const Weights psi, int soft, float *__restrict__ lam,
                                                     double *__restrict__ chibar, double *__restrict__ part,
                                                     int nblk) {
  double acc[LBE_MAX_ELECTRODES];  // psibar
  for (int k = 0; k < LBE_MAX_ELECTRODES; ++k) acc[k] = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    coords32(g, (int)r, x, y, z);
    const uint32_t m = mask[r];
    const int e = id[r];
    if (!e) {
      const double mr = mu[r], pr = phi[r];
      lam[r] += (float)(-P.four_pi_lb * P.z[0] * mr);
      lam[g.N + r] += (float)(-P.four_pi_lb * P.z[1] * mr);
      double dR = psi.c[soft] - pr;  // d R_r / d chi_r
      for (int l = 1; l < kQ; ++l) {
        const uint32_t b = 1u << (l - 1);
        if ((P.selfmask & b) || (m & b)) continue;
        const long long j = link_nbr(g, x, y, z, l);
        dR -= 2.0 * lapc_of(l) * (psi.c[id[j]] - pr);
      }
      chibar[r] += -mr * dR;
    } else {
      const double ps = psi.c[e];
      double mus = -(double)phibar[r], lphi = 0.0, nb = 0.0;
      for (int l = 1; l < kQ; ++l) {
        const uint32_t b = 1u << (l - 1);
        if (P.selfmask & b) continue;
        const long long j = link_nbr(g, x, y, z, l);
        if (j < 0 || j == r) continue;
        const double w = lapc_of(l);
        if (m & b) {
          mus += 2.0 * w * mu[j];
          lphi += 2.0 * w * ((double)phi[j] - ps);
          nb += mu[j] * 2.0 * w * (ps - (double)phi[j]);
        } else {
          lphi += w * (psi.c[id[j]] - ps);
        }
      }
      acc[e - 1] += -mus;
      chibar[r] += mus * lphi - nb;
    }
  }
  block_partials<0, LBE_MAX_ELECTRODES>(acc, part, nblk);
}

// transpose of one flux step: lam_in = nbar^{t+1}, state (q, phi) of time t
// -> nbar^t, phibar^t, Dbar, chibar (openness).  1:1 salt: with
// x = phi_j - phi_r - E.c the two ions see dmu = +x and -x, so one pair
// (e^x - 1, e^-x - 1) serves both.  Per-node sums in FP32, across nodes FP64.
__global__ void __launch_bounds__(kBlock) k_adj_flux(const Geo g, const Phys P, const P32 P3,
                                                     const uint32_t *__restrict__ mask, const uint8_t *__restrict__ id,
                                                     const int64_t *__restrict__ q, const float *__restrict__ phi,
                                                     const Weights psi, const float *__restrict__ lam_in,
                                                     float *__restrict__ lam_out, float *__restrict__ phibar,
                                                     double *__restrict__ chibar, double *__restrict__ part,
                                                     int nblk) {
  const float a0inv = 1.f / (1.f + 2.f * sqrtf(2.f));  // d = D / A0
  const float d0 = (float)P.d[0], d1 = (float)P.d[1];
  const float rb0 = (float)P3.rbd[0], rb1 = (float)P3.rbd[1];
  const float unit = ldexpf(1.f, -kFixBits);
  const int N = (int)g.N;
  double acc[2] = {0.0, 0.0};  // Dbar of the two species
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
    int x, y, z;
    coords32(g, r, x, y, z);
    const uint32_t m = mask[r];
    const int e = id[r];
    if (!e) {
      const Offs o = offsets_of(g, x, y, z);
      const float pr = phi[r];
      const float l0 = lam_in[r], l1 = lam_in[N + r];
      const float nu0 = unit * (float)q[r], nu1 = unit * (float)q[N + r];
      float nb0 = l0, nb1 = l1, pb = 0.f, cb = 0.f, dD0 = 0.f, dD1 = 0.f;
#pragma unroll
      for (int l = 1; l < kQ; ++l) {
        const uint32_t b = 1u << (l - 1);
        if ((P.selfmask & b) || !(m & b)) continue;
        const int j = r + o.at(cx_of(l), cy_of(l), cz_of(l));
        const float il = (float)invlen_of(l);
        float Pp, Mm;
        fp32::em1_pair(phi[j] - pr - (float)P.e_dot_c[l], Pp, Mm);
        const float ep = 1.f + Pp, em = 1.f + Mm;
        // n = rho_b (1 + nu): n' e^dmu - n = rho_b ((nu' - nu) + (1 + nu') (e^dmu - 1))
        const float nuj0 = unit * (float)q[j], nuj1 = unit * (float)q[N + j];
        const float dnu0 = unit * (float)(q[j] - q[r]), dnu1 = unit * (float)(q[N + j] - q[N + r]);
        // species 0 (z = +1): dmu = x
        {
          const float dlam = lam_in[j] - l0;
          const float avg = 0.5f * (1.f + em), br = rb0 * (dnu0 + (1.f + nuj0) * Pp);
          const float J = -d0 * il * avg * br;
          nb0 += dlam * d0 * il * avg;                                                   // dJ/dn_r
          pb -= dlam * (-d0 * il * 0.5f * (rb0 * (1.f + nu0) * em + rb0 * (1.f + nuj0) * ep));  // dJ/dphi_r
          dD0 += dlam * (-a0inv * il * avg * br);                                       // dJ/dD
          cb -= dlam * J;                                                                // openness
        }
        // species 1 (z = -1): dmu = -x
        {
          const float dlam = lam_in[N + j] - l1;
          const float avg = 0.5f * (1.f + ep), br = rb1 * (dnu1 + (1.f + nuj1) * Mm);
          const float J = -d1 * il * avg * br;
          nb1 += dlam * d1 * il * avg;
          pb += dlam * (-d1 * il * 0.5f * (rb1 * (1.f + nu1) * ep + rb1 * (1.f + nuj1) * em));
          dD1 += dlam * (-a0inv * il * avg * br);
          cb -= dlam * J;
        }
      }
      lam_out[r] = nb0;
      lam_out[N + r] = nb1;
      phibar[r] = pb;
      chibar[r] += (double)cb;
      acc[0] += 0.5 * (double)dD0;  // each link is seen from both ends
      acc[1] += 0.5 * (double)dD1;
    } else {
      lam_out[r] = lam_out[N + r] = 0.f;
      phibar[r] = 0.f;
      if (!(m & ((1u << 18) - 1))) continue;
      const Offs o = offsets_of(g, x, y, z);
      const float ps = (float)psi.c[e];
      float cb = 0.f;
#pragma unroll
      for (int l = 1; l < kQ; ++l) {
        const uint32_t b = 1u << (l - 1);
        if ((P.selfmask & b) || !(m & b)) continue;
        const int j = r + o.at(cx_of(l), cy_of(l), cz_of(l));
        const float il = (float)invlen_of(l);
        float Pp, Mm;
        fp32::em1_pair(phi[j] - ps - (float)P.e_dot_c[l], Pp, Mm);
        const float ep = 1.f + Pp, em = 1.f + Mm;
        const float n0 = rb0 * (1.f + unit * (float)q[j]), n1 = rb1 * (1.f + unit * (float)q[N + j]);
        // the flux a link from this node (no ions) to fluid j would carry
        const float J0 = -d0 * il * 0.5f * (1.f + em) * n0 * ep;
        const float J1 = -d1 * il * 0.5f * (1.f + ep) * n1 * em;
        cb -= lam_in[j] * J0 + lam_in[N + j] * J1;
      }
      chibar[r] += (double)cb;
    }
  }
  block_partials<kSlotD, kSlotD + 2>(acc, part, nblk);
}

// t = 0: n^0 = rho_b (1 - chi)
__global__ void __launch_bounds__(kBlock) k_adj_init(long long N, const uint32_t *__restrict__ mask, double rho_b,
                                                     const float *__restrict__ lam, double *__restrict__ chibar,
                                                     double *__restrict__ part, int nblk) {
  double acc[1] = {0.0};  // rho_bbar
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    if (!(mask[r] & kFluidBit)) continue;
    const double s = (double)lam[r] + (double)lam[N + r];
    acc[0] += s;
    chibar[r] += -rho_b * s;
  }
  block_partials<kSlotRho, kSlotRho + 1>(acc, part, nblk);
}

// acc[k] += sum of the block partials of slot k = s0 + block, in block order
__global__ void k_adj_accumulate(const double *__restrict__ part, int nblk, int s0, double *__restrict__ acc) {
  const int k = s0 + blockIdx.x;
  double a = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) a += part[(long long)k * nblk + b];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if (threadIdx.x == 0) acc[k] += a;
}

int afail(lbe_handle *h, int code, const std::string &m) {
  h->err = m;
  return code;
}

#define ACK(h, expr)                                                                                   \
  do {                                                                                                 \
    cudaError_t e_ = (expr);                                                                           \
    if (e_ != cudaSuccess) return afail((h), LBE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// every > 0: uniform checkpoints; every = 0: slots checkpoint slots of the
// binomial schedule (nseg = slots - 1, no segment states)
int adj_alloc(lbe_handle *h, int T, int every, int slots = 0) {
  AdjWork *a = h->adj;
  const long long N = h->geo.N;
  const int nseg = every > 0 ? (T > 0 ? (T + every - 1) / every : 0) : slots - 1;
  const bool same = a && a->N == N && a->nseg == nseg && a->every == every;
  if (!same) {
    adjoint_free(h);
    a = h->adj = new AdjWork();
    a->N = N;
    a->nseg = nseg;
    a->every = every;
    a->nblk = (int)std::min<long long>((N + kBlock - 1) / kBlock, 1184);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
      if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    const size_t ns1 = (size_t)nseg + 1;
    alloc((void **)&a->ck_q, sizeof(int64_t) * 2 * N * ns1);
    alloc((void **)&a->ck_phi, sizeof(double) * N * ns1);
    alloc((void **)&a->ck_prev, sizeof(double) * kHist * N * ns1);
    if (every > 0) {
      alloc((void **)&a->st_q, sizeof(int64_t) * 2 * N * every);
      alloc((void **)&a->st_phi, sizeof(float) * N * every);
    }
    alloc((void **)&a->lam, sizeof(float) * 2 * N);
    alloc((void **)&a->lam2, sizeof(float) * 2 * N);
    alloc((void **)&a->phibar, sizeof(float) * N);
    alloc((void **)&a->mu, sizeof(double) * N);
    alloc((void **)&a->mu_prev, sizeof(double) * N);
    alloc((void **)&a->mu_hi, sizeof(float) * N);
    alloc((void **)&a->mu_lo, sizeof(float) * N);
    alloc((void **)&a->rhs, sizeof(double) * N);
    alloc((void **)&a->chibar, sizeof(double) * N);
    alloc((void **)&a->part, sizeof(double) * kAdjSlots * a->nblk);
    alloc((void **)&a->acc, sizeof(double) * kAdjSlots);
    a->ck_hist.assign(ns1, 0);
    if (e != cudaSuccess) {
      adjoint_free(h);
      return afail(h, LBE_ERR_CUDA, std::string("adjoint: device memory: ") + cudaGetErrorString(e));
    }
  }
  a->T = T;
  a->revolve_slots = every > 0 ? 0 : slots;
  return LBE_OK;
}

// binomial schedule: beta(s, r) = C(s + r, s) steps can be reversed with s
// free slots and r recomputations of each step; the smallest r for n steps,
// and the first checkpoint's distance d (the right part n - d then fits s - 1
// slots with r recomputations, the left part d fits s slots with r - 1)
long long beta(int s, int r) {
  long long b = 1;
  for (int i = 1; i <= s; ++i) {
    b = b * (r + i) / i;  // exact: a binomial coefficient at every i
    if (b > (1LL << 40)) return 1LL << 40;
  }
  return b;
}
int revolve_d(int n, int s) {
  int r = 0;
  while (beta(s, r) < n) ++r;
  const long long right = beta(s - 1, r);
  return (int)std::max<long long>(1, n - std::min<long long>(right, n - 1));
}

// checkpoint k <-> the handle's state (solute, potential, warm-start history)
int save_ck(lbe_handle *h, int k) {
  AdjWork *a = h->adj;
  const long long N = h->geo.N;
  ACK(h, cudaMemcpyAsync(a->ck_q + (size_t)k * 2 * N, h->q, sizeof(int64_t) * 2 * N, cudaMemcpyDeviceToDevice,
                         h->stream));
  ACK(h, cudaMemcpyAsync(a->ck_phi + (size_t)k * N, h->phifx, sizeof(int64_t) * N, cudaMemcpyDeviceToDevice,
                         h->stream));
  ACK(h, cudaMemcpyAsync(a->ck_prev + (size_t)k * kHist * N, h->pw.phi_prev, sizeof(double) * kHist * N,
                         cudaMemcpyDeviceToDevice, h->stream));
  a->ck_hist[k] = (char)h->pw.history;
  return LBE_OK;
}

int load_ck(lbe_handle *h, int k) {
  AdjWork *a = h->adj;
  const long long N = h->geo.N;
  ACK(h, cudaMemcpyAsync(h->q, a->ck_q + (size_t)k * 2 * N, sizeof(int64_t) * 2 * N, cudaMemcpyDeviceToDevice,
                         h->stream));
  ACK(h, cudaMemcpyAsync(h->phifx, a->ck_phi + (size_t)k * N, sizeof(int64_t) * N, cudaMemcpyDeviceToDevice,
                         h->stream));
  ACK(h, cudaMemcpyAsync(h->pw.phi_prev, a->ck_prev + (size_t)k * kHist * N, sizeof(double) * kHist * N,
                         cudaMemcpyDeviceToDevice, h->stream));
  h->pw.history = a->ck_hist[k];
  ACK(h, launch_phi32_from_fx(h));
  return LBE_OK;
}

// adjoint Poisson solve at one time: mu, then nbar, psibar, chibar
int adj_poisson(lbe_handle *h, const float *phi_t, const Weights &psi, int soft) {
  AdjWork *a = h->adj;
  const Geo g = h->geo;
  const int nb = a->nblk;
  k_adj_rhs<<<nb, kBlock, 0, h->stream>>>(g.N, h->mask, a->phibar, a->rhs);
  if (a->nsolved > 0)
    k_adj_extrapolate<<<nb, kBlock, 0, h->stream>>>(g.N, h->mask, a->mu, a->mu_prev, a->nsolved > 1 ? 1 : 0);
  a->nsolved += 1;
  ACK(h, cudaGetLastError());
  // relative 1e-7: below the FP32 resolution of the ion adjoint it feeds;
  // the right-hand side -phibar holds floats: float-float residual
  const int rc = poisson_solve_linear(h, a->rhs, a->mu, 1e-30, 1e-7, a->mu_hi, a->mu_lo);
  if (rc != LBE_OK) return rc;
  k_adj_post<<<nb, kBlock, 0, h->stream>>>(g, h->phys, h->mask, h->id, phi_t, a->phibar, a->mu, psi, soft, a->lam,
                                           a->chibar, a->part, nb);
  k_adj_accumulate<<<LBE_MAX_ELECTRODES, 32, 0, h->stream>>>(a->part, nb, 0, a->acc);
  ACK(h, cudaGetLastError());
  return LBE_OK;
}

// The reverse sweep under the binomial schedule.  The handle's state is
// moved between checkpoint slots and recomputed steps; each backward step
// reads the forward state at its time directly from the handle.
struct RevSweep {
  lbe_handle *h;
  Weights psi;
  int soft;
  long long recomputed = 0, adj_iters = 0;
  double ms_re = 0.0, ms_flux = 0.0, ms_solve = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;

  // CG iterations of the adjoint solves since the last reset (the
  // recomputing steps reset the solver's counters)
  int count() {
    ACK(h, cudaMemcpyAsync(h->pw.ctl_host, h->pw.ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToHost, h->stream));
    ACK(h, cudaStreamSynchronize(h->stream));
    adj_iters += h->pw.ctl_host->total_iters;
    const int status = h->pw.ctl_host->status ? h->pw.ctl_host->status : h->pw.ctl_host->sticky_status;
    if (status) return afail(h, status, "adjoint: Poisson solve failed");
    return LBE_OK;
  }
  int timed(double *acc, int (*f)(RevSweep *, int), int arg) {
    ACK(h, cudaEventRecord(e0, h->stream));
    const int rc = f(this, arg);
    if (rc != LBE_OK) return rc;
    ACK(h, cudaEventRecord(e1, h->stream));
    ACK(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    ACK(h, cudaEventElapsedTime(&ms, e0, e1));
    *acc += ms;
    return LBE_OK;
  }
  static int advance(RevSweep *R, int n) {
    R->recomputed += n;
    return n > 0 ? lbe_step(R->h, n) : LBE_OK;
  }
  static int flux(RevSweep *R, int) {
    AdjWork *a = R->h->adj;
    const int nb = a->nblk;
    k_adj_flux<<<nb, kBlock, 0, R->h->stream>>>(R->h->geo, R->h->phys, R->h->p32, R->h->mask, R->h->id, R->h->q,
                                                R->h->phi32, R->psi, a->lam, a->lam2, a->phibar, a->chibar, a->part,
                                                nb);
    k_adj_accumulate<<<2, 32, 0, R->h->stream>>>(a->part, nb, kSlotD, a->acc);
    ACK(R->h, cudaGetLastError());
    std::swap(a->lam, a->lam2);
    return LBE_OK;
  }
  static int solve(RevSweep *R, int) {
    ACK(R->h, poisson_reset_stats(R->h));
    const int rc = adj_poisson(R->h, R->h->phi32, R->psi, R->soft);
    if (rc != LBE_OK) return rc;
    return R->count();
  }
  // the transposed flux step t -> t+1 and the adjoint solve at time t, from
  // the forward state at t (in the handle)
  int back(int) {
    int rc = timed(&ms_flux, flux, 0);
    if (rc != LBE_OK) return rc;
    return timed(&ms_solve, solve, 0);
  }
  int step(int n) { return timed(&ms_re, advance, n); }

  // Reverse the steps t1-1 .. t0; slot `base` holds x(t0), slots above it
  // are free, s of them usable.  On the first descent (first) the forward
  // pass already stored the next checkpoint in slot base + 1.
  int reverse(int t0, int t1, int base, int s, bool first) {
    const int n = t1 - t0;
    int rc;
    if (n <= 0) return LBE_OK;
    if (n == 1) {
      if ((rc = load_ck(h, base)) != LBE_OK) return rc;
      return back(t0);
    }
    if (s == 0) {  // no free slot: recompute from x(t0) for every step
      for (int t = t1 - 1; t >= t0; --t) {
        if ((rc = load_ck(h, base)) != LBE_OK) return rc;
        if ((rc = step(t - t0)) != LBE_OK) return rc;
        if ((rc = back(t)) != LBE_OK) return rc;
      }
      return LBE_OK;
    }
    const int d = revolve_d(n, s);
    if (!first) {
      if ((rc = load_ck(h, base)) != LBE_OK) return rc;
      if ((rc = step(d)) != LBE_OK) return rc;
      if ((rc = save_ck(h, base + 1)) != LBE_OK) return rc;
    }
    if ((rc = reverse(t0 + d, t1, base + 1, s - 1, first)) != LBE_OK) return rc;
    return reverse(t0, t0 + d, base, s, false);
  }
};

bool adjoint_supported(const lbe_handle *h, std::string *why) {
  const lbe_params &p = h->prm;
  if (p.precision != LBE_FP32) return *why = "adjoint: FP32 form only", false;
  if (p.flow) return *why = "adjoint: solvent at rest only (flow = 0)", false;
  if (!h->p32.salt11 || p.rho_bulk[0] != p.rho_bulk[1])
    return *why = "adjoint: 1:1 salt (z = +1, -1) with one bulk concentration only", false;
  if (!h->have_geometry) return *why = "adjoint: no geometry", false;
  return true;
}

}  // namespace

void adjoint_free(lbe_handle *h) {
  AdjWork *a = h->adj;
  if (!a) return;
  for (cudaEvent_t e : a->ev) cudaEventDestroy(e);
  void *ptrs[] = {a->ck_q, a->ck_phi, a->ck_prev, a->st_q, a->st_phi, a->lam, a->lam2, a->phibar,
                  a->mu,   a->rhs,    a->chibar,  a->part, a->acc, a->mu_prev, a->mu_hi, a->mu_lo};
  for (void *p : ptrs) cudaFree(p);
  delete a;
  h->adj = nullptr;
}

}  // namespace lbe

extern "C" {

int lbe_adjoint_forward(lbe_handle *h, int nsteps, int checkpoint_every, double *q_out) {
  using namespace lbe;
  if (!h) return LBE_ERR_ARG;
  std::string why;
  if (!adjoint_supported(h, &why)) return afail(h, LBE_ERR_STATE, why);
  if (nsteps < 0 || checkpoint_every < 1) return afail(h, LBE_ERR_ARG, "adjoint_forward: bad step counts");
  int rc = adj_alloc(h, nsteps, checkpoint_every);
  if (rc != LBE_OK) return rc;
  AdjWork *a = h->adj;
  a->ready = false;
  rc = lbe_init(h);
  if (rc != LBE_OK) return rc;
  for (int s = 0; s < a->nseg; ++s) {
    rc = save_ck(h, s);
    if (rc != LBE_OK) return rc;
    rc = lbe_step(h, std::min(checkpoint_every, nsteps - s * checkpoint_every));
    if (rc != LBE_OK) return rc;
  }
  rc = save_ck(h, a->nseg);  // time T, restored after a backward pass
  if (rc != LBE_OK) return rc;
  double q[LBE_MAX_ELECTRODES] = {};
  if (h->n_elec) {
    rc = lbe_induced_charge(h, q, 0);
    if (rc != LBE_OK) return rc;
  }
  for (int e = 0; e < h->n_elec; ++e) {
    a->q[e] = q[e];
    if (q_out) q_out[e] = q[e];
  }
  ACK(h, cudaStreamSynchronize(h->stream));
  a->gen = h->gen;
  a->ready = true;
  return LBE_OK;
}

int lbe_adjoint_forward_budget(lbe_handle *h, int nsteps, size_t device_bytes, double *q_out) {
  using namespace lbe;
  if (!h) return LBE_ERR_ARG;
  std::string why;
  if (!adjoint_supported(h, &why)) return afail(h, LBE_ERR_STATE, why);
  if (nsteps < 0) return afail(h, LBE_ERR_ARG, "adjoint_forward_budget: bad step count");
  const size_t N = (size_t)h->geo.N;
  const size_t per_slot = N * (2 * sizeof(int64_t) + sizeof(double) + kHist * sizeof(double));
  const size_t slots = device_bytes / per_slot;
  if (slots < 2) return afail(h, LBE_ERR_ARG, "adjoint_forward_budget: budget below two checkpoints");
  const int nslot = (int)std::min<size_t>(slots, (size_t)nsteps + 2);
  int rc = adj_alloc(h, nsteps, 0, nslot);
  if (rc != LBE_OK) return rc;
  AdjWork *a = h->adj;
  a->ready = false;
  rc = lbe_init(h);
  if (rc != LBE_OK) return rc;
  if ((rc = save_ck(h, 0)) != LBE_OK) return rc;
  // the first descent of the schedule, as the reverse sweep will expect it
  int t0 = 0, s = nslot - 2, k = 0;
  while (nsteps - t0 > 1 && s > 0) {
    const int d = revolve_d(nsteps - t0, s);
    if ((rc = lbe_step(h, d)) != LBE_OK) return rc;
    if ((rc = save_ck(h, k + 1)) != LBE_OK) return rc;
    t0 += d;
    ++k;
    --s;
  }
  if ((rc = lbe_step(h, nsteps - t0)) != LBE_OK) return rc;
  if ((rc = save_ck(h, a->nseg)) != LBE_OK) return rc;  // time T
  double q[LBE_MAX_ELECTRODES] = {};
  if (h->n_elec) {
    rc = lbe_induced_charge(h, q, 0);
    if (rc != LBE_OK) return rc;
  }
  for (int e = 0; e < h->n_elec; ++e) {
    a->q[e] = q[e];
    if (q_out) q_out[e] = q[e];
  }
  ACK(h, cudaStreamSynchronize(h->stream));
  a->gen = h->gen;
  a->ready = true;
  return LBE_OK;
}

int lbe_adjoint_backward(lbe_handle *h, const double *dq, int soft_electrode, lbe_adjoint_grad *out, double *dchi,
                         int dchi_on_device) {
  using namespace lbe;
  if (!h) return LBE_ERR_ARG;
  AdjWork *a = h->adj;
  if (!a || !a->ready || a->gen != h->gen)
    return afail(h, LBE_ERR_STATE, "adjoint_backward: no forward pass (or the state changed since)");
  if (!dq || !out || soft_electrode < 1 || soft_electrode > h->n_elec)
    return afail(h, LBE_ERR_ARG, "adjoint_backward: bad arguments");
  const Geo g = h->geo;
  const long long N = g.N;
  const int nb = a->nblk;
  Weights cq{}, psi{};
  for (int e = 0; e < h->n_elec; ++e) {
    cq.c[e + 1] = dq[e];
    psi.c[e + 1] = h->psi[e];
  }
  cudaStream_t st = h->stream;
  ACK(h, cudaMemsetAsync(a->lam, 0, sizeof(float) * 2 * N, st));
  ACK(h, cudaMemsetAsync(a->mu, 0, sizeof(double) * N, st));
  ACK(h, cudaMemsetAsync(a->mu_prev, 0, sizeof(double) * N, st));
  a->nsolved = 0;
  ACK(h, cudaMemsetAsync(a->chibar, 0, sizeof(double) * N, st));
  ACK(h, cudaMemsetAsync(a->acc, 0, sizeof(double) * kAdjSlots, st));
  // CG iterations of the adjoint solves: the recomputing steps reset the
  // solver's counters, so they are read after each block of adjoint solves
  long long adj_iters = 0;
  auto count = [&]() -> int {
    ACK(h, cudaMemcpyAsync(h->pw.ctl_host, h->pw.ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToHost, st));
    ACK(h, cudaStreamSynchronize(st));
    adj_iters += h->pw.ctl_host->total_iters;
    const int status = h->pw.ctl_host->status ? h->pw.ctl_host->status : h->pw.ctl_host->sticky_status;
    if (status) return afail(h, status, "adjoint: Poisson solve failed");
    return LBE_OK;
  };
  ACK(h, poisson_reset_stats(h));
  // time T (the handle holds the forward pass's final state)
  k_adj_seed<<<nb, kBlock, 0, st>>>(g, h->phys, h->mask, h->id, h->phi32, cq, psi, soft_electrode, a->phibar,
                                    a->chibar);
  ACK(h, cudaGetLastError());
  int rc = adj_poisson(h, h->phi32, psi, soft_electrode);
  if (rc != LBE_OK) return rc;
  if ((rc = count()) != LBE_OK) return rc;
  long long recomputed = 0;
  double ms_re = 0.0, ms_flux = 0.0, ms_solve = 0.0;
  if (a->revolve_slots > 0) {  // binomial schedule
    RevSweep R{h, psi, soft_electrode};
    ACK(h, cudaEventCreate(&R.e0));
    ACK(h, cudaEventCreate(&R.e1));
    rc = R.reverse(0, a->T, 0, a->revolve_slots - 2, true);
    cudaEventDestroy(R.e0);
    cudaEventDestroy(R.e1);
    if (rc != LBE_OK) return rc;
    recomputed = R.recomputed;
    adj_iters += R.adj_iters;
    ms_re = R.ms_re;
    ms_flux = R.ms_flux;
    ms_solve = R.ms_solve;
  }
  while ((int)a->ev.size() < 2 * a->every + 3) {
    cudaEvent_t e;
    ACK(h, cudaEventCreate(&e));
    a->ev.push_back(e);
  }
  for (int s = a->revolve_slots > 0 ? -1 : a->nseg - 1; s >= 0; --s) {
    const int t0 = s * a->every, t1 = std::min(a->T, t0 + a->every);
    ACK(h, cudaEventRecord(a->ev[0], st));
    rc = load_ck(h, s);
    if (rc != LBE_OK) return rc;
    for (int t = t0; t < t1; ++t) {
      ACK(h, cudaMemcpyAsync(a->st_q + (size_t)(t - t0) * 2 * N, h->q, sizeof(int64_t) * 2 * N,
                             cudaMemcpyDeviceToDevice, st));
      ACK(h, cudaMemcpyAsync(a->st_phi + (size_t)(t - t0) * N, h->phi32, sizeof(float) * N, cudaMemcpyDeviceToDevice,
                             st));
      if (t + 1 < t1) {
        rc = lbe_step(h, 1);
        if (rc != LBE_OK) return rc;
        ++recomputed;
      }
    }
    ACK(h, cudaEventRecord(a->ev[1], st));
    ACK(h, poisson_reset_stats(h));
    int k = 2;
    for (int t = t1 - 1; t >= t0; --t) {
      const int64_t *qt = a->st_q + (size_t)(t - t0) * 2 * N;
      const float *pt = a->st_phi + (size_t)(t - t0) * N;
      ACK(h, cudaEventRecord(a->ev[k++], st));
      k_adj_flux<<<nb, kBlock, 0, st>>>(g, h->phys, h->p32, h->mask, h->id, qt, pt, psi, a->lam, a->lam2, a->phibar,
                                        a->chibar, a->part, nb);
      k_adj_accumulate<<<2, 32, 0, st>>>(a->part, nb, kSlotD, a->acc);
      ACK(h, cudaGetLastError());
      ACK(h, cudaEventRecord(a->ev[k++], st));
      std::swap(a->lam, a->lam2);
      rc = adj_poisson(h, pt, psi, soft_electrode);
      if (rc != LBE_OK) return rc;
    }
    ACK(h, cudaEventRecord(a->ev[k], st));
    if ((rc = count()) != LBE_OK) return rc;  // synchronises
    float ms = 0.f;
    ACK(h, cudaEventElapsedTime(&ms, a->ev[0], a->ev[1]));
    ms_re += ms;
    for (int j = 2; j < k; j += 2) {
      ACK(h, cudaEventElapsedTime(&ms, a->ev[j], a->ev[j + 1]));
      ms_flux += ms;
      ACK(h, cudaEventElapsedTime(&ms, a->ev[j + 1], a->ev[j + 2]));
      ms_solve += ms;
    }
  }
  k_adj_init<<<nb, kBlock, 0, st>>>(N, h->mask, h->prm.rho_bulk[0], a->lam, a->chibar, a->part, nb);
  k_adj_accumulate<<<1, 32, 0, st>>>(a->part, nb, kSlotRho, a->acc);
  ACK(h, cudaGetLastError());
  double acc[kAdjSlots];
  ACK(h, cudaMemcpyAsync(acc, a->acc, sizeof(acc), cudaMemcpyDeviceToHost, st));
  if (dchi)
    ACK(h, cudaMemcpyAsync(dchi, a->chibar, sizeof(double) * N,
                           dchi_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  ACK(h, cudaStreamSynchronize(st));
  memset(out, 0, sizeof(*out));
  for (int e = 0; e < h->n_elec; ++e) out->dpsi[e] = acc[e];
  for (int k = 0; k < 2; ++k) out->dD[k] = acc[kSlotD + k];
  out->drho_bulk = acc[kSlotRho];
  out->poisson_iters = adj_iters;
  out->recomputed_steps = recomputed;
  out->recompute_ms = ms_re;
  out->flux_ms = ms_flux;
  out->solve_ms = ms_solve;
  // leave the handle as the forward pass left it
  rc = load_ck(h, a->nseg);
  if (rc != LBE_OK) return rc;
  ACK(h, cudaStreamSynchronize(st));
  h->gen = a->gen;
  return LBE_OK;
}

}  // extern "C"
