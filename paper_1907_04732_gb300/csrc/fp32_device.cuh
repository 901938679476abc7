// Per-node device code of the FP32 form, shared by the single-lattice
// kernels (kernels_fp32.cu) and the batched kernels (batch.cu).  Arrays are
// SoA with component stride N; r is a node's index and o its neighbour
// offsets.
#pragma once

#include <type_traits>

#include "lbe_internal.cuh"

namespace lbe {
namespace fp32 {

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

// Population component offsets: 32-bit while 19 N < 2^31, else 64-bit
// (WIDE; a large lattice or batch passes 2^31 over 19 components).
template <bool WIDE>
using PopIdx = typename std::conditional<WIDE, long long, int>::type;

// pull streaming with halfway bounce-back (see kernels_fp64.cu)
template <bool WIDE>
__device__ __forceinline__ void gather32(int N, int r, const Offs &o, uint32_t m, const float *__restrict__ fin,
                                         float f[kQ]) {
  f[0] = fin[r];
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int io = opp_of(i);
    f[i] = (m & (1u << (io - 1))) ? fin[(PopIdx<WIDE>)i * N + nb_of(o, r, io)] : fin[(PopIdx<WIDE>)io * N + r];
  }
}

// One link of a 1:1 salt (z = +1, -1) from a node with potential phi0 and
// solute nu0 (nu = s q) to its neighbour r2: the flux terms J0, J1 of the two
// species (Eq. LF2, relative form) and the link excess flux gs summed over
// them.  A fixed rounding sequence: evaluated from the other end the link
// gives exactly -J0, -J1, -gs.
__device__ __forceinline__ void link_salt11_nu(const P32 &P, float phi0, float phi2, float ec, float il,
                                               const float nu0[2], const float nu2[2], float &J0, float &J1,
                                               float &gs) {
  const float dphi = __fsub_rn(__fsub_rn(phi2, phi0), ec);
  float P1, M1;
  em1_pair(dphi, P1, M1);
  gs = 0.f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float Pk = k == 0 ? P1 : M1, Mk = k == 0 ? M1 : P1;
    const float nu1 = nu2[k];
    const float a1 = nE(P.rb[k], nu1, Pk), a0 = nE(P.rb[k], nu0[k], Mk);
    const float J = __fsub_rn(tterm(a1, nu1), tterm(a0, nu0[k]));  // t1 - t0, exactly odd under link reversal
    if (k == 0) J0 = J;
    else J1 = J;
    // link excess flux g = j/d + (n' - n)/|c| = -(n' (e^mu - 1) - n (e^-mu - 1))/(2|c|)
    gs = __fmaf_rn(-(il * 0.5f), __fsub_rn(a1, a0), gs);
  }
}
// the same with the neighbour's solute read from q (nu = s q)
__device__ __forceinline__ void link_salt11(const P32 &P, int N, int r2, float phi0, float ec, float il,
                                            const float nu0[2], const int64_t *__restrict__ q,
                                            const float *__restrict__ phi, float &J0, float &J1, float &gs) {
  const float nu2[2] = {__fmul_rn(P.s[0], ll2f(q[r2])), __fmul_rn(P.s[1], ll2f(q[N + r2]))};
  link_salt11_nu(P, phi0, phi[r2], ec, il, nu0, nu2, J0, J1, gs);
}

// The quantised solute update and the force of link i (1:1 salt) from its
// flux terms: dq_k -= round(J_k kq_k), F += c_i gs.
__device__ __forceinline__ void link_apply(const P32 &P, int i, float J0, float J1, float gs, long long dq[2],
                                           float &Fx, float &Fy, float &Fz, bool &over) {
  const float jq0 = __fmul_rn(J0, c2_of(i) == 1 ? P.kq1[0] : P.kq2[0]);
  const float jq1 = __fmul_rn(J1, c2_of(i) == 1 ? P.kq1[1] : P.kq2[1]);
  over |= fabsf(jq0) > 1.0e17f;
  over |= fabsf(jq1) > 1.0e17f;
  dq[0] -= f2ll_rn(jq0);
  dq[1] -= f2ll_rn(jq1);
  Fx += cx_of(i) * gs;
  Fy += cy_of(i) * gs;
  Fz += cz_of(i) * gs;
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
  if (SALT11 && QUANT) {
    const float nu0[2] = {q0f[0], q0f[1]};
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      if (!(m & (1u << (i - 1)))) continue;
      float J0, J1, gs;
      link_salt11(P, N, nb_of(o, r, i), phi0, P.ec[i], (float)invlen_of(i), nu0, q, phi, J0, J1, gs);
      link_apply(P, i, J0, J1, gs, dq, Fx, Fy, Fz, over);
    }
    F[0] = Fx * P.inv_2a0;
    F[1] = Fy * P.inv_2a0;
    F[2] = Fz * P.inv_2a0;
    return;
  }
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
      gs = __fmaf_rn(-(il * 0.5f), __fsub_rn(a1, a0), gs);
    }
    Fx += cx_of(i) * gs;
    Fy += cy_of(i) * gs;
    Fz += cz_of(i) * gs;
  }
  F[0] = Fx * P.inv_2a0;
  F[1] = Fy * P.inv_2a0;
  F[2] = Fz * P.inv_2a0;
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


// BGK + Guo collision and pull streaming with halfway bounce-back at one
// fluid node, given the solvent force F; the velocity is stored
template <bool WIDE>
__device__ __forceinline__ void lb_node(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                        const float *__restrict__ fin, float *__restrict__ fout,
                                        float *__restrict__ u, const float F[3]) {
  float f[kQ];
  gather32<WIDE>(N, r, o, m, fin, f);
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
    fout[(PopIdx<WIDE>)i * N + r] = f[i] - P.omega * (f[i] - (eq_even + eq_odd)) + (src_even + src_odd);
    fout[(PopIdx<WIDE>)io * N + r] = f[io] - P.omega * (f[io] - (eq_even - eq_odd)) + (src_even - src_odd);
  }
}

// Fused step at one fluid node: quantised link fluxes and q* = q - sum Jq,
// solvent force, and (FLOW) BGK + Guo collision with pull streaming.
template <bool FLOW, bool SALT11, bool WIDE>
__device__ __forceinline__ void sweep_node(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                           const float *__restrict__ fin, float *__restrict__ fout,
                                           const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                           const float *__restrict__ phi, float *__restrict__ u, bool &over) {
  long long q0[LBE_MAX_SPECIES], dq[LBE_MAX_SPECIES];
  float q0f[LBE_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    q0[k] = k < P.ns ? q[k * N + r] : 0;
    q0f[k] = k < P.ns ? __fmul_rn(P.s[k], ll2f(q0[k])) : 0.f;  // nu = s q
    dq[k] = 0;
  }
  float F[3];
  ion_links<true, SALT11>(P, N, r, o, m, q, phi, q0, q0f, dq, F, over);
  // compile-time species indices keep q0/dq in registers
#pragma unroll
  for (int k = 0; k < (SALT11 ? 2 : LBE_MAX_SPECIES); ++k)
    if (SALT11 || k < P.ns) qstar[k * N + r] = q0[k] + dq[k];
  if (FLOW) lb_node<WIDE>(P, N, r, o, m, fin, fout, u, F);
}

// Cell-overlap advection at one fluid node (see k_advect32).
__device__ __forceinline__ void advect_node(int ns, int N, int r, const Offs &o, uint32_t m,
                                            const int64_t *__restrict__ qin, const float *__restrict__ u,
                                            int64_t *__restrict__ qout) {
  const float ux = u[r], uy = u[N + r], uz = u[2 * N + r];
  const long long base = 1LL << kFixBits;
  // species loops run to the compile-time bound (guarded by ns) so that acc
  // and totf stay in registers
  long long acc[LBE_MAX_SPECIES];
  float totf[LBE_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    acc[k] = k < ns ? base + qin[k * N + r] : 0;
    totf[k] = ll2f(acc[k]);
  }
  // outgoing (the share is zero outside the octant of u); shares bound for
  // solid neighbours stay
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(dx, dy, dz)))) continue;
    if ((dx && dx * ux <= 0.f) || (dy && dy * uy <= 0.f) || (dz && dz * uz <= 0.f)) continue;
#pragma unroll
    for (int k = 0; k < LBE_MAX_SPECIES; ++k)
      if (k < ns) acc[k] -= share(totf[k], ux, uy, uz, dx, dy, dz);
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
#pragma unroll
    for (int k = 0; k < LBE_MAX_SPECIES; ++k)
      if (k < ns) acc[k] += share(ll2f(base + qin[k * N + s]), vx, vy, vz, dx, dy, dz);
  }
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k)
    if (k < ns) qout[k * N + r] = acc[k] - base;
}

// Warm start of the next solve at fluid node i: the polynomial in time
// through the last history + 1 solutions, one step ahead,
//   history 3: phi <- 4 phi(t) - 6 phi(t-1) + 4 phi(t-2) - phi(t-3)
//   history 2: phi <- 3 phi(t) - 3 phi(t-1) + phi(t-2)
//   history 1: phi <- 2 phi(t) - phi(t-1)
// (the converged potential does not depend on the starting guess).  While an
// electro-osmosis capacitor charges (tolerance 1e-12) the quadratic start is
// 30-300 times closer to the converged potential than the linear one, the
// cubic one another 15 times closer early in the charging and 1.2-3 times
// later.  Its FP32 split follows when hi is given; the history shifts:
// prev = [phi(t), phi(t-1), ...] with component stride N.
__device__ __forceinline__ void extrapolate_node(long long N, long long i, double *__restrict__ phi,
                                                 double *__restrict__ prev, float *__restrict__ hi,
                                                 float *__restrict__ lo, int history) {
  const double v = phi[i], p1 = prev[i];
  if (history > 0) {
    double e;
    if (history == 1) {
      e = 2.0 * v - p1;
    } else if (history == 2) {
      e = prev[N + i] + 3.0 * (v - p1);
    } else {
      const double p2 = prev[N + i], p3 = prev[2 * N + i];
      e = v + 3.0 * (v - p1) - 3.0 * (p1 - p2) + (p2 - p3);
    }
    phi[i] = e;
    if (hi) {  // the FP32 copies follow: the solve may stop at once
      const float h = (float)e;
      hi[i] = h;
      if (lo) lo[i] = (float)(e - (double)h);
    }
  }
#pragma unroll
  for (int k = kHist - 1; k >= 1; --k) prev[k * N + i] = prev[(k - 1) * N + i];
  prev[i] = v;
}

// Error-free sum (Knuth): s + e = a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// 6 lap_mod(phi)(r) for phi = hi + lo (two floats per node), accumulated in
// float-float on the FP32 pipes: per link the difference of the high parts
// is split exactly (two_sum), the low parts and the rounding errors go to the
// error word.  Returns S + E ~ 6 lap to ~2^-46 of the terms; the FP64 form
// of lap_at needs 18 FP64 adds, which are slow on this GPU.
__device__ __forceinline__ void lap6_ff(const Geo &g, int r, int x, int y, int z, uint32_t m,
                                        const float *__restrict__ hi, const float *__restrict__ lo, float &S,
                                        float &E) {
  const Offs o = offsets_of(g, x, y, z);
  const float h0 = hi[r], l0 = lo[r];
  S = 0.f;
  E = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int j = r + o.at(cx_of(i), cy_of(i), cz_of(i));
    const float w = (float)((c2_of(i) == 1 ? 2 : 1) * ((m & (1u << (i - 1))) ? 1 : 2));
    float d, de;
    two_sum(hi[j], -h0, d, de);  // d + de = hi_j - hi_r exactly
    float t, te;
    two_sum(S, w * d, t, te);  // w is a power of two: w d is exact
    S = t;
    E += te + w * (de + (lo[j] - l0));
  }
}

}  // namespace fp32
}  // namespace lbe
