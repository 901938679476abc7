// FP32 lattice kernels of the LBE step ("FP32 deviation" form).
//
// Storage: populations as FP32 deviations df_i = f_i - w_i from the rest
// state (rho = 1, u = 0); solute amounts as int64 fixed point
// n_k = rho_k^bulk + s_k q_k with s_k = rho_k^bulk 2^-40; the potential in
// int64 fixed point (unit 2^-48, the Poisson solve's master copy) plus its
// nearest float, read here.
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
#include "fp32_device.cuh"

namespace lbe {

namespace {

using namespace fp32;

__global__ void k_init32(const Geo g, const P32 P, const uint8_t *__restrict__ id, float *__restrict__ f,
                         int64_t *__restrict__ q, float4 *__restrict__ u) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const bool fl = id[r] == 0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i * g.N + r] = 0.f;
  for (int k = 0; k < P.ns; ++k) q[k * g.N + r] = fl ? 0 : -(1LL << kFixBits);
  u[r] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Link records of a 1:1 salt (fp32::link_record): per fluid node its FP32
// potential and solute deviations, from the state the next sweep reads.
__global__ void __launch_bounds__(kBlock) k_prep32(const Geo g, const P32 P, const float *__restrict__ phi,
                                                   const int64_t *__restrict__ q, float4 *__restrict__ lf) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  // every node's record (a solid node's is never read): the loads need not
  // wait for the mask
  lf[r] = link_record(P, phi[r], q[r], q[g.N + r]);
}

// Fused step kernel of a 1:1 salt: link fluxes from the link records
// (quantised, exactly conserving), solute update q* = q - sum Jq, solvent
// force, and (FLOW) BGK + Guo collision and pull streaming with halfway
// bounce-back, all in FP32 deviations, the populations updated in place
// (one buffer, fin == fout; LAYOUT = POP_AA_EVEN or POP_AA_ODD, the AA
// pattern of fp32_device.cuh: every population slot is read and then
// written by a single node, so the two pointers may alias).  Capped at 64
// registers (four blocks per SM).
template <bool FLOW, int WIDE, int LAYOUT>
__global__ void __launch_bounds__(kBlock, 4) k_sweep32(const Geo g, const P32 P, const uint32_t *__restrict__ mask,
                                                    const float *__restrict__ fin, float *__restrict__ fout,
                                                    const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                                    const float4 *__restrict__ lf, float4 *__restrict__ u,
                                                    int *__restrict__ flag) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) return;
  bool over = false;
  sweep_node_lf<FLOW, WIDE, LAYOUT>(P, N, r, offsets_of(g, x, y, z), m, fin, fout, q, qstar, lf, u, over);
  if (over) atomicOr(flag, 1);
}

// The same for any other salt (several species, valences other than +-1):
// each link evaluated at both ends with a fixed rounding sequence.
template <bool FLOW, int WIDE, int LAYOUT>
__global__ void __launch_bounds__(kBlock) k_sweep32_gen(const Geo g, const P32 P, const uint32_t *__restrict__ mask,
                                                        const float *__restrict__ fin, float *__restrict__ fout,
                                                        const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                                        const float *__restrict__ phi, float4 *__restrict__ u,
                                                        int *__restrict__ flag) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) return;
  bool over = false;
  sweep_node<FLOW, WIDE, LAYOUT>(P, N, r, offsets_of(g, x, y, z), m, fin, fout, q, qstar, phi, u, over);
  if (over) atomicOr(flag, 1);
}

// Cell-overlap advection in fixed point: the share a source hands to a fluid
// neighbour is computed identically by the source (which gives it away) and
// by the target (which collects it), so solute moves in exact integers.  A
// displaced cell only reaches the octant its velocity points to, so a node
// gives to at most 7 neighbours and collects only from neighbours whose
// velocity points at it.  Capped at 48 registers (five blocks per SM): on the
// 64x64x256 electro-osmosis lattice 0.056 ms per step against 0.062 ms at
// the 64 registers the two-species form takes uncapped.
__global__ void __launch_bounds__(kBlock, 5) k_advect32(const Geo g, int ns, const uint32_t *__restrict__ mask,
                                                     const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                                     int64_t *__restrict__ qout, int64_t *__restrict__ phifx,
                                                     int64_t *__restrict__ prev, float *__restrict__ phi32,
                                                     int history) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int k = 0; k < ns; ++k) qout[k * N + r] = qin[k * N + r];
    return;
  }
  if (ns == 2)
    advect_node2(N, r, offsets_of(g, x, y, z), m, qin, u, qout);
  else
    advect_node(ns, N, r, offsets_of(g, x, y, z), m, qin, u, qout);
  // the next solve's warm start (the potential is not read by the advection)
  if (phifx) extrapolate_fx(N, r, phifx, prev, phi32, history);
}

// The FP64 potential (as the API set it) -> fixed point and its float, every
// node; a non-finite value or one beyond kPhiMax raises range flag 4
__global__ void k_phi_from64(const Geo g, const double *__restrict__ phi, int64_t *__restrict__ phifx,
                             float *__restrict__ phi32, int *__restrict__ flag) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  double v = phi[r];
  if (!(fabs(v) < kPhiMax)) {
    atomicOr(flag, 4);
    v = 0.0;
  }
  const long long f = __double2ll_rn(v * 281474976710656.0);  // 2^kPhiFixBits
  phifx[r] = f;
  phi32[r] = fx_to_f(f);
}

// fixed point -> the FP64 copy (exact while |phi| < 2^5, to FP64 rounding beyond)
__global__ void k_phi_to64(const Geo g, const int64_t *__restrict__ phifx, double *__restrict__ phi) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  phi[r] = (double)phifx[r] * (1.0 / 281474976710656.0);
}

__global__ void k_phi32_from_fx(const Geo g, const int64_t *__restrict__ phifx, float *__restrict__ phi32) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  phi32[r] = fx_to_f(phifx[r]);
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
template <int LAYOUT>
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
  gather32<2, false, LAYOUT>(N, r, o, m, fin, f);  // what the next step's collision reads
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
  ion_links<false>(P, N, r, o, m, q, phi, q0, q0f, dq, F, over);
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

#define LAUNCH3(h) make_launch((h)->geo).grid, make_launch((h)->geo).block

}  // namespace

cudaError_t launch_init32(lbe_handle *h) {
  k_init32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->id, h->f32[0], h->q, h->u32);
  h->aa_odd = false;
  return cudaGetLastError();
}

cudaError_t launch_sweep32(lbe_handle *h) {
  const P32 &P = h->p32;
  // 32-bit population offsets while the 19 components fit (pop_idx_kind);
  // the even in-place step of a 1:1 salt takes 64-bit offsets: in that form
  // it compiles without spilling under the 64-register cap (measured on the
  // 64x64x256 electro-osmosis lattice: sweep phase 0.0623 against 0.0633 ms)
  const int wide = pop_idx_kind(h->geo.N);
  const bool flow = h->prm.flow != 0;
  const bool odd = flow && h->aa_odd;  // the populations' in-place step kind
  float *pop = h->f32[0];
  if (P.salt11) {
    k_prep32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, P, h->phi32, h->q, h->lf);
    using Kern = void (*)(const Geo, const P32, const uint32_t *, const float *, float *, const int64_t *, int64_t *,
                          const float4 *, float4 *, int *);
    const Kern k[3][3] = {
        {k_sweep32<false, 0, POP_AA_EVEN>, k_sweep32<false, 1, POP_AA_EVEN>, k_sweep32<false, 2, POP_AA_EVEN>},
        {k_sweep32<true, 0, POP_AA_EVEN>, k_sweep32<true, 1, POP_AA_EVEN>, k_sweep32<true, 2, POP_AA_EVEN>},
        {k_sweep32<true, 0, POP_AA_ODD>, k_sweep32<true, 1, POP_AA_ODD>, k_sweep32<true, 2, POP_AA_ODD>}};
    k[flow + odd][flow && !odd ? 2 : wide]<<<LAUNCH3(h), 0, h->stream>>>(h->geo, P, h->mask, pop, pop, h->q,
                                                                         h->qstar, h->lf, h->u32, h->flag);
  } else {
    using Kern = void (*)(const Geo, const P32, const uint32_t *, const float *, float *, const int64_t *, int64_t *,
                          const float *, float4 *, int *);
    const Kern k[3][3] = {{k_sweep32_gen<false, 0, POP_AA_EVEN>, k_sweep32_gen<false, 1, POP_AA_EVEN>,
                           k_sweep32_gen<false, 2, POP_AA_EVEN>},
                          {k_sweep32_gen<true, 0, POP_AA_EVEN>, k_sweep32_gen<true, 1, POP_AA_EVEN>,
                           k_sweep32_gen<true, 2, POP_AA_EVEN>},
                          {k_sweep32_gen<true, 0, POP_AA_ODD>, k_sweep32_gen<true, 1, POP_AA_ODD>,
                           k_sweep32_gen<true, 2, POP_AA_ODD>}};
    k[flow + odd][wide]<<<LAUNCH3(h), 0, h->stream>>>(h->geo, P, h->mask, pop, pop, h->q, h->qstar, h->phi32,
                                                      h->u32, h->flag);
  }
  if (flow) h->aa_odd = !h->aa_odd;
  return cudaGetLastError();
}

cudaError_t launch_advect32(lbe_handle *h, bool extrapolate) {
  k_advect32<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->prm.nspecies, h->mask, h->qstar, h->u32, h->q,
                                           extrapolate ? h->phifx : nullptr, (int64_t *)h->pw.phi_prev, h->phi32,
                                           h->pw.history);
  if (extrapolate) h->phi64_stale = true;
  return cudaGetLastError();
}

cudaError_t launch_phi_from64(lbe_handle *h) {
  k_phi_from64<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->phi, h->phifx, h->phi32, h->flag);
  h->phi64_stale = false;
  return cudaGetLastError();
}

cudaError_t sync_phi64(lbe_handle *h) {
  if (h->prm.precision != LBE_FP32 || !h->phi64_stale) return cudaSuccess;
  k_phi_to64<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->phifx, h->phi);
  h->phi64_stale = false;
  return cudaGetLastError();
}

cudaError_t launch_phi32_from_fx(lbe_handle *h) {
  k_phi32_from_fx<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->phifx, h->phi32);
  h->phi64_stale = true;
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
  (h->aa_odd ? k_moments32<POP_AA_ODD> : k_moments32<POP_AA_EVEN>)<<<LAUNCH3(h), 0, h->stream>>>(
      h->geo, h->p32, h->prm.flow, h->mask, h->f32[0], h->q, h->phi32, rho_out, u_out, f_out);
  return cudaGetLastError();
}

}  // namespace lbe
