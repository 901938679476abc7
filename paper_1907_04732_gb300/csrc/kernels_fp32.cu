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
#include "lbe_internal.cuh"

namespace lbe {

namespace {

__device__ __forceinline__ long long nbr_i(const Geo &g, int x, int y, int z, int i) {
  return nbr(g, x, y, z, cx_of(i), cy_of(i), cz_of(i));
}

// P = e^x - 1 and M = e^-x - 1.  For |x| <= 1/4 from the Taylor series of
// sinh and cosh - 1 (odd and even parts: P = ch + sh, M = ch - sh), so that
// the pair for -x is exactly (M, P); beyond that from expm1f on x and -x,
// which has the same property.  Truncation error < 1e-10 relative.
__device__ __forceinline__ void em1_pair(float x, float &P, float &M) {
  if (fabsf(x) <= 0.25f) {
    const float x2 = x * x;
    const float sh = x * (1.f + x2 * (1.f / 6.f) * (1.f + x2 * (1.f / 20.f) * (1.f + x2 * (1.f / 42.f))));
    const float ch = x2 * 0.5f * (1.f + x2 * (1.f / 12.f) * (1.f + x2 * (1.f / 30.f) * (1.f + x2 * (1.f / 56.f))));
    P = __fadd_rn(ch, sh);
    M = __fsub_rn(ch, sh);
  } else {
    P = expm1f(x);
    M = expm1f(-x);
  }
}

// t - 2 rho_b for t = n (1 + e^{+-mu}), n = rho_b + s q, E = e^{+-mu} - 1:
//   rho_b E + s q (2 + E), with a fixed rounding sequence
__device__ __forceinline__ float tterm(float rb, float s, long long q, float E) {
  return __fmaf_rn(__fmul_rn(s, (float)q), __fadd_rn(2.f, E), __fmul_rn(rb, E));
}

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

__device__ __forceinline__ void gather32(const Geo &g, long long r, int x, int y, int z, uint32_t m,
                                         const float *__restrict__ fin, float f[kQ]) {
  f[0] = fin[r];
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int io = opp_of(i);
    if (m & (1u << (io - 1)))
      f[i] = fin[i * g.N + nbr_i(g, x, y, z, io)];
    else
      f[i] = fin[io * g.N + r];
  }
}

// Fused step kernel: link fluxes (quantised), solute update q* = q - sum Jq,
// solvent force, and (FLOW) BGK + Guo collision and pull streaming with
// halfway bounce-back, all in FP32 deviations.
template <bool FLOW>
__global__ void __launch_bounds__(kBlock) k_sweep32(const Geo g, const P32 P, const uint32_t *__restrict__ mask,
                                                    const float *__restrict__ fin, float *__restrict__ fout,
                                                    const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                                    const float *__restrict__ phi, float *__restrict__ u,
                                                    int *__restrict__ flag) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) return;
  int x, y, z;
  coords(g, r, x, y, z);
  const float phi0 = phi[r];
  long long q0[LBE_MAX_SPECIES], dq[LBE_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    q0[k] = k < P.ns ? q[k * g.N + r] : 0;
    dq[k] = 0;
  }
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  bool over = false;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    if (!(m & (1u << (i - 1)))) continue;
    const long long r2 = nbr_i(g, x, y, z, i);
    // exactly antisymmetric potential difference along the link
    const float dphi = __fsub_rn(__fsub_rn(phi[r2], phi0), P.ec[i]);
    float P1, M1;
    em1_pair(dphi, P1, M1);
    const float il = (float)invlen_of(i);
    float gs = 0.f;
#pragma unroll
    for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
      if (k >= P.ns) break;
      float Pk, Mk;
      if (P.zi[k] == 1) {
        Pk = P1; Mk = M1;
      } else if (P.zi[k] == -1) {
        Pk = M1; Mk = P1;
      } else {
        em1_pair(__fmul_rn(P.zf[k], dphi), Pk, Mk);
      }
      const long long q1 = q[k * g.N + r2];
      const float X = tterm(P.rb[k], P.s[k], q1, Pk);
      const float Y = tterm(P.rb[k], P.s[k], q0[k], Mk);
      const float J = __fsub_rn(X, Y);  // t1 - t0, exactly odd under link reversal
      const float jq = __fmul_rn(J, c2_of(i) == 1 ? P.kq1[k] : P.kq2[k]);
      over |= fabsf(jq) > 1.0e17f;
      dq[k] -= __float2ll_rn(jq);
      // link excess flux g = j/d + (n' - n)/|c| = (-(t1 - t0)/2 + s (q1 - q0))/|c|
      gs += il * __fmaf_rn(-0.5f, J, P.s[k] * (float)(q1 - q0[k]));
    }
    Fx += cx_of(i) * gs;
    Fy += cy_of(i) * gs;
    Fz += cz_of(i) * gs;
  }
  if (over) atomicOr(flag, 1);
  for (int k = 0; k < P.ns; ++k) qstar[k * g.N + r] = q0[k] + dq[k];
  if (!FLOW) return;
  Fx *= P.inv_2a0;
  Fy *= P.inv_2a0;
  Fz *= P.inv_2a0;

  float f[kQ];
  gather32(g, r, x, y, z, m, fin, f);
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    drho += f[i];
    jx += cx_of(i) * f[i];
    jy += cy_of(i) * f[i];
    jz += cz_of(i) * f[i];
  }
  const float rho = 1.f + drho;
  const float inv_rho = 1.f / rho;
  const float ux = (jx + 0.5f * Fx) * inv_rho, uy = (jy + 0.5f * Fy) * inv_rho, uz = (jz + 0.5f * Fz) * inv_rho;
  u[r] = ux;
  u[g.N + r] = uy;
  u[2 * g.N + r] = uz;
  const float uu = ux * ux + uy * uy + uz * uz;
  const float uF = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float w = (float)w_of(i);
    const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    const float cF = cx_of(i) * Fx + cy_of(i) * Fy + cz_of(i) * Fz;
    const float eq = w * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
    const float src = P.guo * w * (3.f * (cF - uF) + 9.f * cu * cF);
    fout[i * g.N + r] = f[i] - P.omega * (f[i] - eq) + src;
  }
}

// fraction of a unit cell displaced by u that overlaps the cell at offset s
__device__ __forceinline__ float ov(int s, float u) {
  return s == 0 ? 1.f - fabsf(u) : (s > 0 ? fmaxf(u, 0.f) : fmaxf(-u, 0.f));
}

__device__ __forceinline__ int dir_bit(int dx, int dy, int dz) {
  if (dx != 0 && dy != 0 && dz != 0) return corner_bit(dx, dy, dz);
#pragma unroll
  for (int i = 1; i < kQ; ++i)
    if (cx_of(i) == dx && cy_of(i) == dy && cz_of(i) == dz) return i - 1;
  return -1;
}

// integer share of a node's solute (in fixed-point units, total amount
// 2^40 + q) that its displaced cell hands to the neighbour at offset s
__device__ __forceinline__ long long share(long long total, float ux, float uy, float uz, int sx, int sy, int sz) {
  const float w = ov(sx, ux) * ov(sy, uy) * ov(sz, uz);
  return (long long)__float2ll_rn(__fmul_rn(w, (float)total));
}

// Cell-overlap advection in fixed point: the share a source hands to a fluid
// neighbour is computed identically by the source (which gives it away) and
// by the target (which collects it), so solute is moved in exact integers.
__global__ void __launch_bounds__(kBlock) k_advect32(const Geo g, int ns, const uint32_t *__restrict__ mask,
                                                     const int64_t *__restrict__ qin, const float *__restrict__ u,
                                                     int64_t *__restrict__ qout) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int k = 0; k < ns; ++k) qout[k * g.N + r] = qin[k * g.N + r];
    return;
  }
  int x, y, z;
  coords(g, r, x, y, z);
  const float ux = u[r], uy = u[g.N + r], uz = u[2 * g.N + r];
  const long long base = 1LL << kFixBits;
  long long acc[LBE_MAX_SPECIES], own[LBE_MAX_SPECIES];
  for (int k = 0; k < ns; ++k) {
    own[k] = base + qin[k * g.N + r];
    acc[k] = own[k];
  }
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        // outgoing share to the neighbour at +s, if it is fluid
        if (m & (1u << dir_bit(dx, dy, dz))) {
          for (int k = 0; k < ns; ++k) acc[k] -= share(own[k], ux, uy, uz, dx, dy, dz);
        }
        // incoming share from the neighbour at -s, if it is fluid
        if (m & (1u << dir_bit(-dx, -dy, -dz))) {
          const long long s = nbr(g, x, y, z, -dx, -dy, -dz);
          const float sx = u[s], sy = u[g.N + s], sz = u[2 * g.N + s];
          for (int k = 0; k < ns; ++k) acc[k] += share(base + qin[k * g.N + s], sx, sy, sz, dx, dy, dz);
        }
      }
  for (int k = 0; k < ns; ++k) qout[k * g.N + r] = acc[k] - base;
}

// output conversions
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

__global__ void k_moments32(const Geo g, const P32 P, int flow, const uint32_t *__restrict__ mask,
                            const float *__restrict__ fin, const int64_t *__restrict__ q,
                            const float *__restrict__ phi, double *__restrict__ rho_out,
                            double *__restrict__ u_out, double *__restrict__ f_out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    if (rho_out) rho_out[r] = 0.0;
    if (u_out) u_out[r] = u_out[g.N + r] = u_out[2 * g.N + r] = 0.0;
    if (f_out)
      for (int i = 0; i < kQ; ++i) f_out[i * g.N + r] = 0.0;
    return;
  }
  int x, y, z;
  coords(g, r, x, y, z);
  float f[kQ];
  gather32(g, r, x, y, z, m, fin, f);
  if (f_out) {
    for (int i = 0; i < kQ; ++i) f_out[i * g.N + r] = w_of(i) + (double)f[i];
    return;
  }
  // solvent force of the current state (same expressions as k_sweep32)
  const float phi0 = phi[r];
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  for (int i = 1; i < kQ; ++i) {
    if (!(m & (1u << (i - 1)))) continue;
    const long long r2 = nbr_i(g, x, y, z, i);
    const float dphi = __fsub_rn(__fsub_rn(phi[r2], phi0), P.ec[i]);
    float P1, M1;
    em1_pair(dphi, P1, M1);
    float gs = 0.f;
    for (int k = 0; k < P.ns; ++k) {
      float Pk, Mk;
      if (P.zi[k] == 1) { Pk = P1; Mk = M1; }
      else if (P.zi[k] == -1) { Pk = M1; Mk = P1; }
      else em1_pair(__fmul_rn(P.zf[k], dphi), Pk, Mk);
      const long long q1 = q[k * g.N + r2], q0 = q[k * g.N + r];
      const float J = __fsub_rn(tterm(P.rb[k], P.s[k], q1, Pk), tterm(P.rb[k], P.s[k], q0, Mk));
      gs += (float)invlen_of(i) * __fmaf_rn(-0.5f, J, P.s[k] * (float)(q1 - q0));
    }
    Fx += cx_of(i) * gs;
    Fy += cy_of(i) * gs;
    Fz += cz_of(i) * gs;
  }
  Fx *= P.inv_2a0;
  Fy *= P.inv_2a0;
  Fz *= P.inv_2a0;
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
    u_out[r] = flow ? (jx + 0.5 * Fx) / rho : 0.0;
    u_out[g.N + r] = flow ? (jy + 0.5 * Fy) / rho : 0.0;
    u_out[2 * g.N + r] = flow ? (jz + 0.5 * Fz) / rho : 0.0;
  }
}

inline unsigned grid_for(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

}  // namespace

cudaError_t launch_init32(lbe_handle *h) {
  k_init32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->id, h->f32[h->cur], h->q, h->u32);
  return cudaGetLastError();
}

cudaError_t launch_sweep32(lbe_handle *h) {
  const int nxt = h->cur ^ 1;
  if (h->prm.flow)
    k_sweep32<true><<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->mask, h->f32[h->cur],
                                                                   h->f32[nxt], h->q, h->qstar, h->phi32,
                                                                   h->u32, h->flag);
  else
    k_sweep32<false><<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->mask, h->f32[h->cur],
                                                                    h->f32[nxt], h->q, h->qstar, h->phi32,
                                                                    h->u32, h->flag);
  if (h->prm.flow) h->cur = nxt;
  return cudaGetLastError();
}

cudaError_t launch_advect32(lbe_handle *h) {
  k_advect32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->prm.nspecies, h->mask, h->qstar, h->u32, h->q);
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
  k_moments32<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->p32, h->prm.flow, h->mask, h->f32[h->cur],
                                                             h->q, h->phi32, rho_out, u_out, f_out);
  return cudaGetLastError();
}

}  // namespace lbe
