// FP32 lattice kernels of the LBE step ("FP32 deviation" form).
//
// Storage: populations as FP32 deviations df_i = f_i - w_i from the rest
// state (rho = 1, u = 0); solute amounts as int64 fixed point
// n_k = rho_k^bulk + s_k q_k with s_k = rho_k^bulk 2^-40; the potential as an
// FP64 master copy (Poisson) plus an FP32 copy read here.
//
// Arithmetic is FP32.  The link flux of Eq. LF2 is evaluated so that the
// value computed at either end of a link is exactly opposite, and is then
// quantised to the fixed-point unit before it updates q: the total solute
// amount of every species is conserved exactly (integer sums), as the link
// flux method conserves it in exact arithmetic (Sec. "Lattice Boltzmann
// Electrokinetics").
//
// No FP64 instruction runs in these kernels: 64-bit integers are converted
// through their 32-bit halves (the 64-bit conversion instructions use the FP64
// pipe, which is narrow on this GPU).
#include <stdlib.h>

#include "fp32_device.cuh"

namespace lbe {

namespace {

using namespace fp32;

__global__ void k_init32(const Geo g, const P32 P, const uint8_t *__restrict__ id, float *__restrict__ f,
                         int64_t *__restrict__ q, float *__restrict__ u) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const bool fl = id[r] == 0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i * g.N + r] = 0.f;
  for (int k = 0; k < P.ns; ++k) q[k * g.N + r] = fl ? 0 : -(1LL << kFixBits);
  u[r] = u[g.N + r] = u[2 * g.N + r] = 0.f;
}

// Fused step kernel: link fluxes (quantised), solute update q* = q - sum Jq,
// solvent force, and (FLOW) BGK + Guo collision and pull streaming with
// halfway bounce-back, all in FP32 deviations.
template <bool FLOW, bool SALT11, bool WIDE>
__global__ void __launch_bounds__(kBlock) k_sweep32(const Geo g, const P32 P, const uint32_t *__restrict__ mask,
                                                    const float *__restrict__ fin, float *__restrict__ fout,
                                                    const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                                    const float *__restrict__ phi, float *__restrict__ u,
                                                    int *__restrict__ flag) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) return;
  bool over = false;
  sweep_node<FLOW, SALT11, WIDE>(P, N, r, offsets_of(g, x, y, z), m, fin, fout, q, qstar, phi, u, over);
  if (over) atomicOr(flag, 1);
}

// Link-sharing form of the fused sweep (1:1 salt, flow on, 32-bit
// population offsets; LBE_SWEEP_SHARED=1 selects it).  Every link is
// evaluated once, by its lower end: a node owns its links to +x, +y, (+x,+y),
// (-x,+y) and the five to the plane above.  A block covers a kTX x kTY tile
// of an x-y plane and marches along z through kZC planes.  Each plane's
// potential, solute (nu = s q) and link mask are staged once in shared memory
// for the tile and a one-node halo; per plane the block evaluates the links
// owned by the tile and the halo from the staged values into shared-memory
// records, and each node then takes its 18 links in the per-node kernel's
// order, a link owned by a neighbour with its record negated (the evaluation
// is exactly antisymmetric): the results are bitwise those of k_sweep32.
// The records of the links into a plane from the plane below are kept in
// registers by the nodes that take them before the records are rewritten.
namespace shared_links {
constexpr int kTX = 32, kTY = 8, kZC = 8, kThreads = kTX * kTY;
constexpr int kEX = kTX + 2, kEY = kTY + 2, kE = kEX * kEY;  // staged region: x0-1..x0+kTX, y0-1..y0+kTY
constexpr int kPI = kEX * (kTY + 1);                        // in-plane link producers: rows y0-1..y0+kTY-1
constexpr int kPU = kE;                                     // up-link producers: the whole staged region
constexpr int kNI = 4, kNU = 5;

__host__ __device__ constexpr int in_dx(int s) { return s == 0 ? 1 : (s == 1 ? 0 : (s == 2 ? 1 : -1)); }
__host__ __device__ constexpr int in_dy(int s) { return s == 0 ? 0 : 1; }
__host__ __device__ constexpr int up_dx(int s) { return s == 1 ? 1 : (s == 2 ? -1 : 0); }
__host__ __device__ constexpr int up_dy(int s) { return s == 3 ? 1 : (s == 4 ? -1 : 0); }
__host__ __device__ constexpr int qidx(int dx, int dy, int dz) {
  for (int i = 1; i < kQ; ++i)
    if (cx_of(i) == dx && cy_of(i) == dy && cz_of(i) == dz) return i;
  return 0;
}
__host__ __device__ constexpr int in_slot(int dx, int dy, int dz) {
  for (int s = 0; s < kNI; ++s)
    if (dz == 0 && in_dx(s) == dx && in_dy(s) == dy) return s;
  return -1;
}
__host__ __device__ constexpr int up_slot(int dx, int dy, int dz) {
  for (int s = 0; s < kNU; ++s)
    if (dz == 1 && up_dx(s) == dx && up_dy(s) == dy) return s;
  return -1;
}
__device__ __forceinline__ int in_q(int s) {
  return s == 0 ? qidx(1, 0, 0) : (s == 1 ? qidx(0, 1, 0) : (s == 2 ? qidx(1, 1, 0) : qidx(-1, 1, 0)));
}
__device__ __forceinline__ int up_q(int s) {
  return s == 0 ? qidx(0, 0, 1)
                : (s == 1 ? qidx(1, 0, 1) : (s == 2 ? qidx(-1, 0, 1) : (s == 3 ? qidx(0, 1, 1) : qidx(0, -1, 1))));
}
// coordinate along an axis of n nodes: wrapped (as often as needed: the
// staged region may be wider than a periodic axis) or -1 outside a
// non-periodic one
__device__ __forceinline__ int wrapc(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  c %= n;
  return c < 0 ? c + n : c;
}

struct Plane {  // one staged plane
  float phi[kE], nu0[kE], nu1[kE];
  uint32_t mask[kE];
};
struct Smem {
  Plane pl[2];
  float rin[3 * kNI * kPI];  // (J0, J1, gs) of the in-plane links, [c][slot][producer]
  float rup[3 * kNU * kPU];  // the same for the links to the next plane
};

__device__ __forceinline__ void stage(const Geo &g, const P32 &P, const uint32_t *__restrict__ mask,
                                      const int64_t *__restrict__ q, const float *__restrict__ phi, int x0, int y0,
                                      int z, Plane &pl) {
  const int N = (int)g.N;
  const int zc = wrapc(z, g.nz, g.pz);
  for (int e = threadIdx.y * kTX + threadIdx.x; e < kE; e += kThreads) {
    const int x = wrapc(x0 - 1 + e % kEX, g.nx, g.px), y = wrapc(y0 - 1 + e / kEX, g.ny, g.py);
    if (x >= 0 && y >= 0 && zc >= 0) {
      const int r = x + g.nx * (y + g.ny * zc);
      pl.mask[e] = mask[r];
      pl.phi[e] = phi[r];
      pl.nu0[e] = __fmul_rn(P.s[0], ll2f(q[r]));
      pl.nu1[e] = __fmul_rn(P.s[1], ll2f(q[N + r]));
    } else {
      pl.mask[e] = 0u;  // outside a non-periodic face: no links
      pl.phi[e] = pl.nu0[e] = pl.nu1[e] = 0.f;
    }
  }
}

// records of the links owned by the producers of plane a (in-plane: into a
// itself; UP: into plane b above); a record whose far end lies outside the
// staged region is never taken and left zero
template <bool UP>
__device__ __forceinline__ void produce(const P32 &P, const Plane &a, const Plane &b, float *__restrict__ rec) {
  constexpr int nslot = UP ? kNU : kNI, np = UP ? kPU : kPI;
  for (int t = threadIdx.y * kTX + threadIdx.x; t < nslot * np; t += kThreads) {
    const int s = t / np, p = t - s * np;
    const int ex = p % kEX, ey = p / kEX;
    const int dx = UP ? up_dx(s) : in_dx(s), dy = UP ? up_dy(s) : in_dy(s);
    const int ex2 = ex + dx, ey2 = ey + dy;
    float J0 = 0.f, J1 = 0.f, gs = 0.f;
    if (ex2 >= 0 && ex2 < kEX && ey2 >= 0 && ey2 < kEY) {
      const uint32_t m = a.mask[p];
      const int i = UP ? up_q(s) : in_q(s);
      if ((m & kFluidBit) && (m & (1u << (i - 1)))) {
        const Plane &o = UP ? b : a;
        const int p2 = ey2 * kEX + ex2;
        const float nu0[2] = {a.nu0[p], a.nu1[p]}, nu2[2] = {o.nu0[p2], o.nu1[p2]};
        const float il = (dx != 0) + (dy != 0) + (UP ? 1 : 0) == 1 ? (float)invlen_of(qidx(1, 0, 0))
                                                                     : (float)invlen_of(qidx(1, 1, 0));
        link_salt11_nu(P, a.phi[p], o.phi[p2], P.ec[i], il, nu0, nu2, J0, J1, gs);
      }
    }
    rec[(0 * nslot + s) * np + p] = J0;
    rec[(1 * nslot + s) * np + p] = J1;
    rec[(2 * nslot + s) * np + p] = gs;
  }
}
}  // namespace shared_links

__global__ void __launch_bounds__(shared_links::kThreads)
    k_sweep32_shared(const Geo g, const P32 P, const uint32_t *__restrict__ mask, const float *__restrict__ fin,
                     float *__restrict__ fout, const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                     const float *__restrict__ phi, float *__restrict__ u, int *__restrict__ flag) {
  using namespace shared_links;
  __shared__ Smem sm;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * kZC;
  const int z1 = min(z0 + kZC, g.nz);
  const int tx = threadIdx.x, ty = threadIdx.y, x = x0 + tx, y = y0 + ty, N = (int)g.N;
  const int pown = (ty + 1) * kEX + (tx + 1);  // this node in the staged region and the producer grids
  bool over = false;
  int cur = 1;  // slot of plane z; the other holds plane z - 1, then z + 1
  stage(g, P, mask, q, phi, x0, y0, z0 - 1, sm.pl[0]);
  stage(g, P, mask, q, phi, x0, y0, z0, sm.pl[1]);
  __syncthreads();
  produce<true>(P, sm.pl[0], sm.pl[1], sm.rup);  // links into the first plane from below
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    // this node's links from the plane below (records about to be rewritten)
    float dn[kNU][3];
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      if (cz_of(i) != -1) continue;
      const int s = up_slot(-cx_of(i), -cy_of(i), 1), k = s, pp = pown + cy_of(i) * kEX + cx_of(i);
      dn[k][0] = sm.rup[(0 * kNU + s) * kPU + pp];
      dn[k][1] = sm.rup[(1 * kNU + s) * kPU + pp];
      dn[k][2] = sm.rup[(2 * kNU + s) * kPU + pp];
    }
    __syncthreads();
    stage(g, P, mask, q, phi, x0, y0, z + 1, sm.pl[cur ^ 1]);  // plane z - 1 is no longer needed
    __syncthreads();
    produce<false>(P, sm.pl[cur], sm.pl[cur], sm.rin);
    produce<true>(P, sm.pl[cur], sm.pl[cur ^ 1], sm.rup);
    __syncthreads();
    if (x < g.nx && y < g.ny) {
      const int r = x + g.nx * (y + g.ny * z);
      const uint32_t m = sm.pl[cur].mask[pown];
      if (m & kFluidBit) {
        long long dq[2] = {0, 0};
        float Fx = 0.f, Fy = 0.f, Fz = 0.f;
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
          if (!(m & (1u << (i - 1)))) continue;
          const int dx = cx_of(i), dy = cy_of(i), dz = cz_of(i);
          float J0, J1, gs;
          if (in_slot(dx, dy, dz) >= 0) {  // owned, in-plane
            const int s = in_slot(dx, dy, dz);
            J0 = sm.rin[(0 * kNI + s) * kPI + pown];
            J1 = sm.rin[(1 * kNI + s) * kPI + pown];
            gs = sm.rin[(2 * kNI + s) * kPI + pown];
          } else if (up_slot(dx, dy, dz) >= 0) {  // owned, to the plane above
            const int s = up_slot(dx, dy, dz);
            J0 = sm.rup[(0 * kNU + s) * kPU + pown];
            J1 = sm.rup[(1 * kNU + s) * kPU + pown];
            gs = sm.rup[(2 * kNU + s) * kPU + pown];
          } else if (dz == 0) {  // owned by the in-plane neighbour at +c
            const int s = in_slot(-dx, -dy, 0), pp = pown + dy * kEX + dx;
            J0 = -sm.rin[(0 * kNI + s) * kPI + pp];
            J1 = -sm.rin[(1 * kNI + s) * kPI + pp];
            gs = -sm.rin[(2 * kNI + s) * kPI + pp];
          } else {  // owned by the neighbour in the plane below
            const int s = up_slot(-dx, -dy, 1);
            J0 = -dn[s][0];
            J1 = -dn[s][1];
            gs = -dn[s][2];
          }
          link_apply(P, i, J0, J1, gs, dq, Fx, Fy, Fz, over);
        }
        qstar[r] = q[r] + dq[0];
        qstar[N + r] = q[N + r] + dq[1];
        const float F[3] = {Fx * P.inv_2a0, Fy * P.inv_2a0, Fz * P.inv_2a0};
        lb_node<false>(P, N, r, offsets_of(g, x, y, z), m, fin, fout, u, F);
      }
    }
    cur ^= 1;
  }
  if (over) atomicOr(flag, 1);
}

// Cell-overlap advection in fixed point: the share a source hands to a fluid
// neighbour is computed identically by the source (which gives it away) and
// by the target (which collects it), so solute moves in exact integers.  A
// displaced cell only reaches the octant its velocity points to, so a node
// gives to at most 7 neighbours and collects only from neighbours whose
// velocity points at it.
__global__ void __launch_bounds__(kBlock) k_advect32(const Geo g, int ns, const uint32_t *__restrict__ mask,
                                                     const int64_t *__restrict__ qin, const float *__restrict__ u,
                                                     int64_t *__restrict__ qout, double *__restrict__ phi,
                                                     double *__restrict__ prev, float *__restrict__ phi32,
                                                     float *__restrict__ phi_lo, int history) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int k = 0; k < ns; ++k) qout[k * N + r] = qin[k * N + r];
    return;
  }
  advect_node(ns, N, r, offsets_of(g, x, y, z), m, qin, u, qout);
  // the next solve's warm start (phi is not read by the advection)
  if (phi) extrapolate_node(N, r, phi, prev, phi32, phi_lo, history);
}

__global__ void k_n_to_double(const Geo g, const P32 P, const int64_t *__restrict__ q, const uint32_t *__restrict__ mask,
                              double *__restrict__ out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const bool fl = mask[r] & kFluidBit;
  for (int k = 0; k < P.ns; ++k)
    out[k * g.N + r] = fl ? P.rbd[k] + P.sd[k] * (double)q[k * g.N + r] : 0.0;
}

__global__ void k_n_from_double(const Geo g, const P32 P, const double *__restrict__ n,
                                const uint32_t *__restrict__ mask, int64_t *__restrict__ q, int *__restrict__ flag) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const bool fl = mask[r] & kFluidBit;
  for (int k = 0; k < P.ns; ++k) {
    if (!fl) {
      q[k * g.N + r] = -(1LL << kFixBits);
      continue;
    }
    const double v = (n[k * g.N + r] - P.rbd[k]) / P.sd[k];
    if (!(fabs(v) < 4.0e18)) {
      atomicOr(flag, 2);
      q[k * g.N + r] = 0;
    } else {
      q[k * g.N + r] = __double2ll_rn(v);
    }
  }
}

// density, velocity (current state) or populations, as FP64
__global__ void k_moments32(const Geo g, const P32 P, int flow, const uint32_t *__restrict__ mask,
                            const float *__restrict__ fin, const int64_t *__restrict__ q,
                            const float *__restrict__ phi, double *__restrict__ rho_out,
                            double *__restrict__ u_out, double *__restrict__ f_out) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    if (rho_out) rho_out[r] = 0.0;
    if (u_out) u_out[r] = u_out[N + r] = u_out[2 * N + r] = 0.0;
    if (f_out)
      for (int i = 0; i < kQ; ++i) f_out[(long long)i * N + r] = 0.0;
    return;
  }
  const Offs o = offsets_of(g, x, y, z);
  float f[kQ];
  gather32<true>(N, r, o, m, fin, f);
  if (f_out) {
    for (int i = 0; i < kQ; ++i) f_out[(long long)i * N + r] = w_of(i) + (double)f[i];
    return;
  }
  long long q0[LBE_MAX_SPECIES], dq[LBE_MAX_SPECIES];
  float q0f[LBE_MAX_SPECIES];
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    q0[k] = k < P.ns ? q[k * N + r] : 0;
    q0f[k] = k < P.ns ? __fmul_rn(P.s[k], ll2f(q0[k])) : 0.f;  // nu = s q
    dq[k] = 0;
  }
  float F[3];
  bool over = false;
  ion_links<false, false>(P, N, r, o, m, q, phi, q0, q0f, dq, F, over);
  double drho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < kQ; ++i) {
    drho += f[i];
    jx += cx_of(i) * (double)f[i];
    jy += cy_of(i) * (double)f[i];
    jz += cz_of(i) * (double)f[i];
  }
  const double rho = 1.0 + drho;
  if (rho_out) rho_out[r] = rho;
  if (u_out) {
    u_out[r] = flow ? (jx + 0.5 * F[0]) / rho : 0.0;
    u_out[N + r] = flow ? (jy + 0.5 * F[1]) / rho : 0.0;
    u_out[2 * N + r] = flow ? (jz + 0.5 * F[2]) / rho : 0.0;
  }
}

inline unsigned grid_for(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

// the link-sharing sweep (k_sweep32_shared) when LBE_SWEEP_SHARED=1 (read at
// every launch, so that one process can compare both kernels)
inline bool shared_sweep_enabled() {
  const char *e = getenv("LBE_SWEEP_SHARED");
  return e && e[0] == '1';
}
#define LAUNCH3(h) make_launch((h)->geo).grid, make_launch((h)->geo).block

}  // namespace

cudaError_t launch_init32(lbe_handle *h) {
  k_init32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->id, h->f32[h->cur], h->q, h->u32);
  return cudaGetLastError();
}

cudaError_t launch_sweep32(lbe_handle *h) {
  const int nxt = h->cur ^ 1;
  const P32 &P = h->p32;
  const bool salt11 = P.ns == 2 && P.zi[0] == 1 && P.zi[1] == -1;
  using Kern = void (*)(const Geo, const P32, const uint32_t *, const float *, float *, const int64_t *, int64_t *,
                        const float *, float *, int *);
  // 32-bit population offsets while the 19 components fit
  const bool wide = (long long)kQ * h->geo.N >= (1LL << 31);
  if (h->prm.flow && salt11 && !wide && shared_sweep_enabled()) {
    const Geo &g = h->geo;
    using namespace shared_links;
    const dim3 grid((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kZC - 1) / kZC);
    k_sweep32_shared<<<grid, dim3(kTX, kTY), 0, h->stream>>>(g, P, h->mask, h->f32[h->cur], h->f32[nxt], h->q,
                                                             h->qstar, h->phi32, h->u32, h->flag);
    h->cur = nxt;
    return cudaGetLastError();
  }
  Kern kern = wide ? (h->prm.flow ? (salt11 ? k_sweep32<true, true, true> : k_sweep32<true, false, true>)
                                  : (salt11 ? k_sweep32<false, true, true> : k_sweep32<false, false, true>))
                   : (h->prm.flow ? (salt11 ? k_sweep32<true, true, false> : k_sweep32<true, false, false>)
                                  : (salt11 ? k_sweep32<false, true, false> : k_sweep32<false, false, false>));
  kern<<<LAUNCH3(h), 0, h->stream>>>(h->geo, P, h->mask, h->f32[h->cur], h->f32[nxt], h->q, h->qstar, h->phi32,
                                     h->u32, h->flag);
  if (h->prm.flow) h->cur = nxt;
  return cudaGetLastError();
}

cudaError_t launch_advect32(lbe_handle *h, bool extrapolate) {
  k_advect32<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->prm.nspecies, h->mask, h->qstar, h->u32, h->q,
                                           extrapolate ? h->phi : nullptr, h->pw.phi_prev, h->phi32, h->phi_lo,
                                           h->pw.history);
  return cudaGetLastError();
}

cudaError_t launch_n_to_double(lbe_handle *h, double *out) {
  k_n_to_double<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->q, h->mask, out);
  return cudaGetLastError();
}

cudaError_t launch_n_from_double(lbe_handle *h, const double *n) {
  k_n_from_double<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, n, h->mask, h->q, h->flag);
  return cudaGetLastError();
}

cudaError_t launch_moments32(lbe_handle *h, double *rho_out, double *u_out, double *f_out) {
  k_moments32<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->p32, h->prm.flow, h->mask, h->f32[h->cur],
                                                             h->q, h->phi32, rho_out, u_out, f_out);
  return cudaGetLastError();
}

}  // namespace lbe
