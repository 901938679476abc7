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
#include "lbe_internal.cuh"

namespace lbe {

namespace {

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

// 64-bit integer <-> float with 32-bit conversions only.  Deterministic, and
// f2ll_rn(-x) = -f2ll_rn(x).
__device__ __forceinline__ float ll2f(long long v) {
  const int lo = (int)v;
  if ((long long)lo == v) return (float)lo;  // fits 32 bits: one conversion
  return __fmaf_rn((float)(int)(v >> 32), 4294967296.f, (float)(unsigned)v);
}
// nearest integer (ties to even) of x, |x| < 2^62
__device__ __forceinline__ long long f2ll_rn(float x) {
  const float r = rintf(x);
  if (fabsf(r) < 2147483648.f) return (long long)__float2int_rn(r);
  const float hi = floorf(r * (1.f / 4294967296.f));
  const float lo = r - hi * 4294967296.f;  // exact: a multiple of ulp(r) below 2^32
  return ((long long)__float2int_rz(hi) << 32) + (long long)__float2uint_rz(lo);
}

// For a link end with solute n = rho_b + nu (nu = s q) and E = e^{+-mu} - 1:
//   a = n E = rho_b E + nu E,   t - 2 rho_b = a + 2 nu   (t = n (1 + e^{+-mu}))
// with a fixed rounding sequence, so that both ends of a link compute the
// same values.
__device__ __forceinline__ float nE(float rb, float nu, float E) { return __fmaf_rn(nu, E, __fmul_rn(rb, E)); }
__device__ __forceinline__ float tterm(float a, float nu) { return __fmaf_rn(2.f, nu, a); }

__device__ __forceinline__ int nb_of(const Offs &o, int r, int i) { return r + o.at(cx_of(i), cy_of(i), cz_of(i)); }

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

// pull streaming with halfway bounce-back (see kernels_fp64.cu)
__device__ __forceinline__ void gather32(int N, int r, const Offs &o, uint32_t m, const float *__restrict__ fin,
                                         float f[kQ]) {
  f[0] = fin[r];
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int io = opp_of(i);
    f[i] = (m & (1u << (io - 1))) ? fin[i * N + nb_of(o, r, io)] : fin[io * N + r];
  }
}

// Ion part of the step at one fluid node: quantised link fluxes -> dq, and
// the solvent force from the link excess fluxes.
template <bool QUANT, bool SALT11>
__device__ __forceinline__ void ion_links(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                          const int64_t *__restrict__ q, const float *__restrict__ phi,
                                          const long long q0[LBE_MAX_SPECIES], const float q0f[LBE_MAX_SPECIES],  // q0f: nu
                                          long long dq[LBE_MAX_SPECIES], float F[3], bool &over) {
  const float phi0 = phi[r];
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    if (!(m & (1u << (i - 1)))) continue;
    const int r2 = nb_of(o, r, i);
    // exactly antisymmetric potential difference along the link
    const float dphi = __fsub_rn(__fsub_rn(phi[r2], phi0), P.ec[i]);
    float P1, M1;
    em1_pair(dphi, P1, M1);
    const float il = (float)invlen_of(i);
    float gs = 0.f;
#pragma unroll
    for (int k = 0; k < (SALT11 ? 2 : LBE_MAX_SPECIES); ++k) {
      if (!SALT11 && k >= P.ns) break;
      float Pk, Mk;
      if (SALT11) {  // z = +1, -1
        Pk = k == 0 ? P1 : M1;
        Mk = k == 0 ? M1 : P1;
      } else if (P.zi[k] == 1) {
        Pk = P1;
        Mk = M1;
      } else if (P.zi[k] == -1) {
        Pk = M1;
        Mk = P1;
      } else {
        em1_pair(__fmul_rn(P.zf[k], dphi), Pk, Mk);
      }
      const float nu1 = __fmul_rn(P.s[k], ll2f(q[k * N + r2]));
      const float a1 = nE(P.rb[k], nu1, Pk), a0 = nE(P.rb[k], q0f[k], Mk);
      const float J = __fsub_rn(tterm(a1, nu1), tterm(a0, q0f[k]));  // t1 - t0, exactly odd under link reversal
      if (QUANT) {
        const float jq = __fmul_rn(J, c2_of(i) == 1 ? P.kq1[k] : P.kq2[k]);
        over |= fabsf(jq) > 1.0e17f;
        dq[k] -= f2ll_rn(jq);
      }
      // link excess flux g = j/d + (n' - n)/|c| = -(n' (e^mu - 1) - n (e^-mu - 1))/(2|c|)
      gs -= il * 0.5f * (a1 - a0);
    }
    Fx += cx_of(i) * gs;
    Fy += cy_of(i) * gs;
    Fz += cz_of(i) * gs;
  }
  F[0] = Fx * P.inv_2a0;
  F[1] = Fy * P.inv_2a0;
  F[2] = Fz * P.inv_2a0;
}

// Fused step kernel: link fluxes (quantised), solute update q* = q - sum Jq,
// solvent force, and (FLOW) BGK + Guo collision and pull streaming with
// halfway bounce-back, all in FP32 deviations.
template <bool FLOW, bool SALT11>
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
  const Offs o = offsets_of(g, x, y, z);
  long long q0[LBE_MAX_SPECIES], dq[LBE_MAX_SPECIES];
  float q0f[LBE_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    q0[k] = k < P.ns ? q[k * N + r] : 0;
    q0f[k] = k < P.ns ? __fmul_rn(P.s[k], ll2f(q0[k])) : 0.f;  // nu = s q
    dq[k] = 0;
  }
  float F[3];
  bool over = false;
  ion_links<true, SALT11>(P, N, r, o, m, q, phi, q0, q0f, dq, F, over);
  if (over) atomicOr(flag, 1);
  for (int k = 0; k < (SALT11 ? 2 : P.ns); ++k) qstar[k * N + r] = q0[k] + dq[k];
  if (!FLOW) return;

  float f[kQ];
  gather32(N, r, o, m, fin, f);
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
  const float ux = (jx + 0.5f * F[0]) * inv_rho, uy = (jy + 0.5f * F[1]) * inv_rho, uz = (jz + 0.5f * F[2]) * inv_rho;
  u[r] = ux;
  u[N + r] = uy;
  u[2 * N + r] = uz;
  const float uu = ux * ux + uy * uy + uz * uz;
  const float uF = ux * F[0] + uy * F[1] + uz * F[2];
  // BGK + Guo forcing; c_{i+9} = -c_i, so each opposite pair shares the even
  // part of the equilibrium and of the source and flips the odd part
  {
    const float w = (float)w_of(0);
    const float eq = w * (drho - rho * 1.5f * uu);
    const float src = -P.guo * w * 3.f * uF;
    fout[r] = f[0] - P.omega * (f[0] - eq) + src;
  }
#pragma unroll
  for (int i = 1; i <= 9; ++i) {
    const float w = (float)w_of(i);
    const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    const float cF = cx_of(i) * F[0] + cy_of(i) * F[1] + cz_of(i) * F[2];
    const float eq_even = w * (drho + rho * (4.5f * cu * cu - 1.5f * uu));
    const float eq_odd = w * rho * 3.f * cu;
    const float src_even = P.guo * w * (9.f * cu * cF - 3.f * uF);
    const float src_odd = P.guo * w * 3.f * cF;
    const int io = i + 9;
    fout[i * N + r] = f[i] - P.omega * (f[i] - (eq_even + eq_odd)) + (src_even + src_odd);
    fout[io * N + r] = f[io] - P.omega * (f[io] - (eq_even - eq_odd)) + (src_even - src_odd);
  }
}

// fraction of a unit cell displaced by u that overlaps the cell at offset s
__device__ __forceinline__ float ov(int s, float u) {
  return s == 0 ? 1.f - fabsf(u) : (s > 0 ? fmaxf(u, 0.f) : fmaxf(-u, 0.f));
}

__host__ __device__ constexpr int dir_bit(int dx, int dy, int dz) {
  if (dx != 0 && dy != 0 && dz != 0) return corner_bit(dx, dy, dz);
  for (int i = 1; i < kQ; ++i)
    if (cx_of(i) == dx && cy_of(i) == dy && cz_of(i) == dz) return i - 1;
  return -1;
}

// integer share (fixed-point units) of a node's total solute 2^40 + q that its
// displaced cell hands to the neighbour at offset s
__device__ __forceinline__ long long share(float totf, float ux, float uy, float uz, int sx, int sy, int sz) {
  const float w = ov(sx, ux) * ov(sy, uy) * ov(sz, uz);
  return w == 0.f ? 0LL : f2ll_rn(__fmul_rn(w, totf));
}

// Cell-overlap advection in fixed point: the share a source hands to a fluid
// neighbour is computed identically by the source (which gives it away) and
// by the target (which collects it), so solute moves in exact integers.  A
// displaced cell only reaches the octant its velocity points to, so a node
// gives to at most 7 neighbours and collects only from neighbours whose
// velocity points at it.
__global__ void __launch_bounds__(kBlock) k_advect32(const Geo g, int ns, const uint32_t *__restrict__ mask,
                                                     const int64_t *__restrict__ qin, const float *__restrict__ u,
                                                     int64_t *__restrict__ qout) {
  int x, y, z;
  long long rl;
  if (!node_of(g, 1, 0, x, y, z, rl)) return;
  const int r = (int)rl, N = (int)g.N;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int k = 0; k < ns; ++k) qout[k * N + r] = qin[k * N + r];
    return;
  }
  const Offs o = offsets_of(g, x, y, z);
  const float ux = u[r], uy = u[N + r], uz = u[2 * N + r];
  const long long base = 1LL << kFixBits;
  long long acc[LBE_MAX_SPECIES];
  float totf[LBE_MAX_SPECIES];
  for (int k = 0; k < ns; ++k) {
    acc[k] = base + qin[k * N + r];
    totf[k] = ll2f(acc[k]);
  }
  // outgoing (the share is zero outside the octant of u); shares bound for
  // solid neighbours stay
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(dx, dy, dz)))) continue;
    if ((dx && dx * ux <= 0.f) || (dy && dy * uy <= 0.f) || (dz && dz * uz <= 0.f)) continue;
    for (int k = 0; k < ns; ++k) acc[k] -= share(totf[k], ux, uy, uz, dx, dy, dz);
  }
  // incoming from every fluid neighbour whose cell reaches r: the source at
  // r - s gives along +s
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(-dx, -dy, -dz)))) continue;
    const int s = r + o.at(-dx, -dy, -dz);
    const float vx = u[s], vy = u[N + s], vz = u[2 * N + s];
    const float w = ov(dx, vx) * ov(dy, vy) * ov(dz, vz);
    if (w == 0.f) continue;
    for (int k = 0; k < ns; ++k) acc[k] += share(ll2f(base + qin[k * N + s]), vx, vy, vz, dx, dy, dz);
  }
  for (int k = 0; k < ns; ++k) qout[k * N + r] = acc[k] - base;
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
      for (int i = 0; i < kQ; ++i) f_out[i * N + r] = 0.0;
    return;
  }
  const Offs o = offsets_of(g, x, y, z);
  float f[kQ];
  gather32(N, r, o, m, fin, f);
  if (f_out) {
    for (int i = 0; i < kQ; ++i) f_out[i * N + r] = w_of(i) + (double)f[i];
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
  Kern kern = h->prm.flow ? (salt11 ? k_sweep32<true, true> : k_sweep32<true, false>)
                          : (salt11 ? k_sweep32<false, true> : k_sweep32<false, false>);
  kern<<<LAUNCH3(h), 0, h->stream>>>(h->geo, P, h->mask, h->f32[h->cur], h->f32[nxt], h->q, h->qstar, h->phi32,
                                     h->u32, h->flag);
  if (h->prm.flow) h->cur = nxt;
  return cudaGetLastError();
}

cudaError_t launch_advect32(lbe_handle *h) {
  k_advect32<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->prm.nspecies, h->mask, h->qstar, h->u32, h->q);
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
