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

// Population component offsets (WIDE): 0 signed 32-bit while 19 N < 2^31,
// 1 unsigned 32-bit while 19 N < 2^32 (the same address arithmetic, one
// more bit: a large lattice or batch), 2 64-bit beyond.
template <int WIDE>
using PopIdx = typename std::conditional<WIDE == 0, int,
                                         typename std::conditional<WIDE == 1, unsigned, long long>::type>::type;
inline int pop_idx_kind(long long N) {
  return 19LL * N < (1LL << 31) ? 0 : (19LL * N < (1LL << 32) ? 1 : 2);
}

// Population layouts of a step, with halfway bounce-back at links to solid
// (bit i-1 of the node mask m clear: x + c_i is solid or outside the box).
//   POP_PULL: two buffers; the step reads the previous step's post-collision
//     values, f_i(x) = fin[i][x - c_i] (bounced back: fin[opp i][x]), and
//     writes its own to fout[i][x] (the batched form).
//   POP_AA_EVEN / POP_AA_ODD: one buffer A updated in place, two kinds of
//     step in turn (the AA pattern of Bailey, Myre, Walsh, Lilja and Saad,
//     2009).  An even step reads f_i(x) = A[i][x] and writes f*_i to
//     A[opp i][x]; an odd step reads f_i(x) = A[opp i][x - c_i] (bounced
//     back: A[i][x]) and writes f*_i to A[i][x + c_i] (bounced back:
//     A[opp i][x]).  Each slot is read, then written, by one node of a step.
// ALL: every link joins fluid (no bounce-back to select).
enum PopLayout { POP_PULL = 0, POP_AA_EVEN = 1, POP_AA_ODD = 2 };

template <int WIDE, bool ALL = false, int LAYOUT = POP_PULL>
__device__ __forceinline__ void gather32(int N, int r, const Offs &o, uint32_t m, const float *__restrict__ fin,
                                         float f[kQ]) {
  f[0] = fin[r];
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int io = opp_of(i);
    const bool in = ALL || (m & (1u << (io - 1)));  // x - c_i is fluid
    if (LAYOUT == POP_PULL)
      f[i] = in ? fin[(PopIdx<WIDE>)i * (PopIdx<WIDE>)N + (PopIdx<WIDE>)nb_of(o, r, io)] : fin[(PopIdx<WIDE>)io * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r];
    else if (LAYOUT == POP_AA_EVEN)
      f[i] = fin[(PopIdx<WIDE>)i * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r];
    else
      f[i] = in ? fin[(PopIdx<WIDE>)io * (PopIdx<WIDE>)N + (PopIdx<WIDE>)nb_of(o, r, io)] : fin[(PopIdx<WIDE>)i * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r];
  }
}

// where post-collision population i of node r goes (i >= 1)
template <int WIDE, bool ALL, int LAYOUT>
__device__ __forceinline__ void put32(int N, int r, const Offs &o, uint32_t m, int i, float v,
                                      float *__restrict__ fout) {
  const int io = opp_of(i);
  if (LAYOUT == POP_PULL)
    fout[(PopIdx<WIDE>)i * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r] = v;
  else if (LAYOUT == POP_AA_EVEN)
    fout[(PopIdx<WIDE>)io * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r] = v;
  else if (ALL || (m & (1u << (i - 1))))
    fout[(PopIdx<WIDE>)i * (PopIdx<WIDE>)N + (PopIdx<WIDE>)nb_of(o, r, i)] = v;
  else
    fout[(PopIdx<WIDE>)io * (PopIdx<WIDE>)N + (PopIdx<WIDE>)r] = v;
}

// ---------------------------------------------------------------------------
// Link records of a 1:1 salt (z = +1, -1): one float4 per fluid node,
// (nu_+, nu_-, phi, 0) with nu = s q, written before each sweep so that the
// link loop reads one record per neighbour instead of converting its 64-bit
// solute amounts.  The two species' values come first, as one aligned pair
// of registers for the paired arithmetic of link_pair.
__device__ __forceinline__ float4 link_record(const P32 &P, float phi, long long q0, long long q1) {
  return make_float4(__fmul_rn(P.s[0], ll2f(q0)), __fmul_rn(P.s[1], ll2f(q1)), phi, 0.f);
}

// Paired FP32 arithmetic (one instruction for two lanes on this GPU), each
// lane rounded exactly as the scalar __fadd_rn / __fmul_rn / __fmaf_rn: the
// two species of a 1:1 salt go through a link's flux terms together.
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 lo_pair(const float4 &v) { return make_float2(v.x, v.y); }

// sinh x and cosh x - 1 from expm1f, for the rare link with |x| > 1/4 (a
// call, so that the common path does not carry it)
static __device__ __noinline__ float2 shch_wide(float x) {
  const float ep = expm1f(x), em = expm1f(-x);
  return make_float2(__fmul_rn(0.5f, __fsub_rn(ep, em)), __fmul_rn(0.5f, __fadd_rn(ep, em)));
}

// Flux terms of both species on the link from its owner a to b (Eq. LF2 in
// the relative form), with x = dmu_+ = phi_b - phi_a - E.c (dmu_- = -x):
//   A_k = n_b (e^{dmu} - 1) - n_a (e^{-dmu} - 1) = S_k sinh(dmu) + D_k (cosh(dmu) - 1)
//   J_k = n_b (1 + e^{dmu}) - n_a (1 + e^{-dmu}) = 2 D_k + A_k
// with S = n_a + n_b, D = n_b - n_a (j = -d J/(2|c|); A is the link excess
// flux of the force up to the factor -1/(2|c|)).  sinh and
// cosh - 1 come from their Taylor series for |x| <= 1/4 (relative error
// below 5e-8) and from expm1f beyond.  Every link is evaluated in this one
// orientation (a = the end from which it points along one of c_1..c_9), by
// both of its end nodes from the same records: the two are bitwise equal.
// The species (+, -) are the two lanes of J = (J_+, J_-) and A = (A_+, A_-);
// rb2 = (2 rho_b+, 2 rho_b-).
__device__ __forceinline__ void link_pair(float2 rb2, const float4 &ra, const float4 &rb, float ec, float2 &J,
                                          float2 &A) {
  const float x = __fsub_rn(__fsub_rn(rb.z, ra.z), ec);
  float sh, ch;
  if (fabsf(x) <= 0.25f) {
    const float x2 = __fmul_rn(x, x);
    sh = __fmul_rn(x, __fmaf_rn(x2, __fmaf_rn(x2, 1.f / 120.f, 1.f / 6.f), 1.f));
    ch = __fmul_rn(x2, __fmaf_rn(x2, 1.f / 24.f, 0.5f));
  } else {
    const float2 w = shch_wide(x);
    sh = w.x;
    ch = w.y;
  }
  const float2 na = lo_pair(ra), nb = lo_pair(rb);
  const float2 D = sub2_rn(nb, na);
  const float2 S = __fadd2_rn(rb2, __fadd2_rn(na, nb));
  // A_+ = S_+ sh + D_+ ch, A_- = -S_- sh + D_- ch (z = -1 flips dmu)
  A = __ffma2_rn(S, make_float2(sh, -sh), __fmul2_rn(D, make_float2(ch, ch)));
  J = __ffma2_rn(make_float2(2.f, 2.f), D, A);
}

// Rounding a link's fluxes x = (x_0, x_1) of the two species (fixed-point
// units, |x| < 2^44) to integers and adding them to (SIGN > 0) or
// subtracting them from (SIGN < 0) two 64-bit amounts, each kept as two
// 32-bit sums hi 2^22 + lo, with FP32 and integer adds only (no conversion
// instructions): per lane h = round(x 2^-22) read off the float grid of unit
// spacing at 1.5 2^23 (kMagic), lo = x - h 2^22 (exact), l = round(lo)
// likewise.  The sums carry kMagicBits per term, removed once per node
// (mod 2^32).  Both roundings are round-half-even, an odd function of x, so
// a link's two ends move exactly opposite amounts.
constexpr float kMagic = 12582912.f;  // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;
template <int SIGN>
__device__ __forceinline__ void acc_round(float2 x, unsigned &ah0, unsigned &al0, unsigned &ah1, unsigned &al1) {
  const float2 mg = make_float2(kMagic, kMagic);
  const float2 h = __ffma2_rn(x, make_float2(2.384185791015625e-07f, 2.384185791015625e-07f), mg);  // 2^-22
  const float2 lo = __ffma2_rn(sub2_rn(h, mg), make_float2(-4194304.f, -4194304.f), x);  // x - (h - M) 2^22
  const float2 l = __fadd2_rn(lo, mg);
  if (SIGN > 0) {
    ah0 += (unsigned)__float_as_int(h.x);
    ah1 += (unsigned)__float_as_int(h.y);
    al0 += (unsigned)__float_as_int(l.x);
    al1 += (unsigned)__float_as_int(l.y);
  } else {
    ah0 -= (unsigned)__float_as_int(h.x);
    ah1 -= (unsigned)__float_as_int(h.y);
    al0 -= (unsigned)__float_as_int(l.x);
    al1 -= (unsigned)__float_as_int(l.y);
  }
}
// the 64-bit amount of two sums after net = (#added - #subtracted) terms
__device__ __forceinline__ long long acc_value(unsigned ah, unsigned al, int net) {
  const unsigned off = (unsigned)net * kMagicBits;
  return (long long)(int)(ah - off) * 4194304LL + (long long)(int)(al - off);
}

// Ion part of the step at one fluid node, any salt (the general form; a 1:1
// salt takes sweep_node_lf): link fluxes evaluated at both ends with a fixed
// rounding sequence (the potential difference is exactly antisymmetric and
// em1_pair(-x) = (M, P) for em1_pair(x) = (P, M)), quantised (QUANT) into dq,
// and the solvent force from the link excess fluxes.
template <bool QUANT>
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
    for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
      if (k >= P.ns) break;
      float Pk, Mk;
      if (P.zi[k] == 1) {
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
        over |= !(fabsf(jq) <= 1.0e17f);  // also catches NaN
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


// Velocity record of a fluid node for the advection: (ux, uy, uz, code),
// code holding which components are positive (bits 0, 2, 4 for x, y, z)
// and negative (bits 1, 3, 5).  A node's displaced cell reaches its
// neighbour at offset s exactly when every nonzero s_a has the sign of u_a
// (|u| < 1), i.e. when code contains cell_bits(s).
__device__ __forceinline__ int octant_code(float ux, float uy, float uz) {
  return (ux > 0.f) | ((ux < 0.f) << 1) | ((uy > 0.f) << 2) | ((uy < 0.f) << 3) | ((uz > 0.f) << 4) |
         ((uz < 0.f) << 5);
}
__host__ __device__ constexpr int cell_bits(int dx, int dy, int dz) {
  return (dx > 0 ? 1 : 0) | (dx < 0 ? 2 : 0) | (dy > 0 ? 4 : 0) | (dy < 0 ? 8 : 0) | (dz > 0 ? 16 : 0) |
         (dz < 0 ? 32 : 0);
}

// BGK + Guo collision and pull streaming with halfway bounce-back at one
// fluid node, given the solvent force F; the velocity is stored.  A density
// deviation of 1/2 or more (or a non-finite one) raises the range flag.
// In deviations df = f - w (Eq. LBpop with the second-order equilibrium and
// Guo's source, reading R4), c_{i+9} = -c_i pairs share the even parts:
//   df'_i = (1 - omega) df_i + E_even +- E_odd,
//   E_even = w [omega (drho + rho (4.5 cu^2 - 1.5 uu)) + guo (9 cu cF - 3 uF)]
//   E_odd  = w [3 omega rho cu + 3 guo cF]
template <int WIDE, bool ALL = false, int LAYOUT = POP_PULL>
__device__ __forceinline__ void lb_collide(const P32 &P, int N, int r, const Offs &o, uint32_t m, const float f[kQ],
                                           float *__restrict__ fout, float4 *__restrict__ u, const float F[3],
                                           bool &over) {
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    drho += f[i];
    jx += cx_of(i) * f[i];
    jy += cy_of(i) * f[i];
    jz += cz_of(i) * f[i];
  }
  over |= !(fabsf(drho) < 0.5f);
  const float rho = 1.f + drho;
  const float inv_rho = 1.f / rho;
  const float ux = (jx + 0.5f * F[0]) * inv_rho, uy = (jy + 0.5f * F[1]) * inv_rho, uz = (jz + 0.5f * F[2]) * inv_rho;
  u[r] = make_float4(ux, uy, uz, __int_as_float(octant_code(ux, uy, uz)));
  const float uu = ux * ux + uy * uy + uz * uz;
  const float uF = ux * F[0] + uy * F[1] + uz * F[2];
  const float om = P.omega, g = P.guo, keep = 1.f - om;
  // w-independent parts per node
  const float base = om * (drho - 1.5f * rho * uu) - 3.f * g * uF;  // E_even / w at cu = cF = 0
  const float b2 = 4.5f * om * rho, d2 = 3.f * om * rho;
  fout[r] = keep * f[0] + (float)w_of(0) * base;
#pragma unroll
  for (int i = 1; i <= 9; ++i) {
    const float w = (float)w_of(i);
    const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    const float cF = cx_of(i) * F[0] + cy_of(i) * F[1] + cz_of(i) * F[2];
    const float ee = w * (base + cu * (b2 * cu + 9.f * g * cF));
    const float eo = w * (d2 * cu + 3.f * g * cF);
    const int io = i + 9;
    put32<WIDE, ALL, LAYOUT>(N, r, o, m, i, keep * f[i] + (ee + eo), fout);
    put32<WIDE, ALL, LAYOUT>(N, r, o, m, io, keep * f[io] + (ee - eo), fout);
  }
}
template <int WIDE, bool ALL = false, int LAYOUT = POP_PULL>
__device__ __forceinline__ void lb_node(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                        const float *__restrict__ fin, float *__restrict__ fout,
                                        float4 *__restrict__ u, const float F[3], bool &over) {
  float f[kQ];
  gather32<WIDE, ALL, LAYOUT>(N, r, o, m, fin, f);
  lb_collide<WIDE, ALL, LAYOUT>(P, N, r, o, m, f, fout, u, F, over);
}

// Fused step at one fluid node, any salt: quantised link fluxes and
// q* = q - sum Jq, solvent force, and (FLOW) BGK + Guo collision with pull
// streaming.
template <bool FLOW, int WIDE, int LAYOUT = POP_PULL>
__device__ __forceinline__ void sweep_node(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                           const float *__restrict__ fin, float *__restrict__ fout,
                                           const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                           const float *__restrict__ phi, float4 *__restrict__ u, bool &over) {
  long long q0[LBE_MAX_SPECIES], dq[LBE_MAX_SPECIES];
  float q0f[LBE_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k) {
    q0[k] = k < P.ns ? q[k * N + r] : 0;
    q0f[k] = k < P.ns ? __fmul_rn(P.s[k], ll2f(q0[k])) : 0.f;  // nu = s q
    dq[k] = 0;
  }
  float F[3];
  ion_links<true>(P, N, r, o, m, q, phi, q0, q0f, dq, F, over);
  // compile-time species indices keep q0/dq in registers
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k)
    if (k < P.ns) qstar[k * N + r] = q0[k] + dq[k];
  if (FLOW) lb_node<WIDE, false, LAYOUT>(P, N, r, o, m, fin, fout, u, F, over);
}

// Fused step at one fluid node of a 1:1 salt from the link records lf
// (link_record): per link the flux terms of both species (link_pair, in the
// link's one orientation), their fixed-point rounding (owner end subtracts,
// the other end adds: exact conservation), the force from the link excess
// fluxes, then (FLOW) BGK + Guo collision with streaming in the given
// population layout.
template <bool FLOW, int WIDE, bool ALL, int LAYOUT>
__device__ __forceinline__ void sweep_node_lf_(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                              const float *__restrict__ fin, float *__restrict__ fout,
                                              const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                              const float4 *__restrict__ lf, float4 *__restrict__ u, bool &over) {
  // PULL (the batched form) reads the populations before the link loop, so
  // that their loads are in flight during the link arithmetic; the in-place
  // layouts read them after it (measured: the early read spills 56-112 B
  // under the 64-register cap and took 0.077 ms against 0.065)
  constexpr bool kEarly = LAYOUT == POP_PULL;
  float f[kQ];
  if (FLOW && kEarly) gather32<WIDE, ALL, LAYOUT>(N, r, o, m, fin, f);
  const float4 self = lf[r];
  const float2 rb2 = make_float2(2.f * P.rb[0], 2.f * P.rb[1]);
  const float2 kq1 = make_float2(P.kq1[0], P.kq1[1]), kq2 = make_float2(P.kq2[0], P.kq2[1]);
  unsigned ah0 = 0u, al0 = 0u, ah1 = 0u, al1 = 0u;
  float2 sq = make_float2(0.f, 0.f);
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    if (!ALL && !(m & (1u << (i - 1)))) continue;
    const float4 nb = lf[nb_of(o, r, i)];
    const bool mine = i <= 9;  // this node owns the link (c_i among c_1..c_9)
    const int d = mine ? i : opp_of(i);
    float2 J, A;
    link_pair(rb2, mine ? self : nb, mine ? nb : self, P.ec[d], J, A);
    const float2 jq = __fmul2_rn(J, c2_of(d) == 1 ? kq1 : kq2);
    sq = __ffma2_rn(jq, jq, sq);
    if (mine)
      acc_round<-1>(jq, ah0, al0, ah1, al1);
    else
      acc_round<1>(jq, ah0, al0, ah1, al1);
    if (FLOW) {
      // link excess flux g = -(A_+ + A_-)/(2|c|) along c_d; both ends take
      // c_d g (from b it is -g along -c_d)
      const float gs = (-0.5f * (float)invlen_of(d)) * (A.x + A.y);
      Fx += cx_of(d) * gs;
      Fy += cy_of(d) * gs;
      Fz += cz_of(d) * gs;
    }
  }
  // every |x| < 2^43 keeps acc_round exact (the sum of squares bounds each
  // link's value); a NaN fails the test too
  over |= !(sq.x + sq.y < 6.4e25f);
  const int net = __popc(m & 0x3FE00u) - __popc(m & 0x1FFu);  // received - owned links
  qstar[r] = q[r] + acc_value(ah0, al0, net);
  qstar[N + r] = q[N + r] + acc_value(ah1, al1, net);
  if (FLOW) {
    const float F[3] = {Fx * P.inv_2a0, Fy * P.inv_2a0, Fz * P.inv_2a0};
    if (!kEarly) gather32<WIDE, ALL, LAYOUT>(N, r, o, m, fin, f);
    lb_collide<WIDE, ALL, LAYOUT>(P, N, r, o, m, f, fout, u, F, over);
  }
}
// the same; a node whose 18 links all join fluid (most of a lattice) takes
// a form without the per-link mask tests
template <bool FLOW, int WIDE, int LAYOUT = POP_PULL>
__device__ __forceinline__ void sweep_node_lf(const P32 &P, int N, int r, const Offs &o, uint32_t m,
                                              const float *__restrict__ fin, float *__restrict__ fout,
                                              const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                              const float4 *__restrict__ lf, float4 *__restrict__ u, bool &over) {
  if ((m & 0x3FFFFu) == 0x3FFFFu)
    sweep_node_lf_<FLOW, WIDE, true, LAYOUT>(P, N, r, o, m, fin, fout, q, qstar, lf, u, over);
  else
    sweep_node_lf_<FLOW, WIDE, false, LAYOUT>(P, N, r, o, m, fin, fout, q, qstar, lf, u, over);
}

// Cell-overlap advection at one fluid node (see k_advect32), from the
// velocity records (octant_code): a neighbour's record is read once and its
// code tells whether its displaced cell reaches this node; only those
// neighbours' solute is read and shared.
__device__ __forceinline__ void advect_node(int ns, int N, int r, const Offs &o, uint32_t m,
                                            const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                            int64_t *__restrict__ qout) {
  const float4 v0 = u[r];
  const int code0 = __float_as_int(v0.w);
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
    if ((code0 & cell_bits(dx, dy, dz)) != cell_bits(dx, dy, dz)) continue;
#pragma unroll
    for (int k = 0; k < LBE_MAX_SPECIES; ++k)
      if (k < ns) acc[k] -= share(totf[k], v0.x, v0.y, v0.z, dx, dy, dz);
  }
  // incoming from every fluid neighbour whose cell reaches r: the source at
  // r - s gives along +s
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(-dx, -dy, -dz)))) continue;
    const int s = r + o.at(-dx, -dy, -dz);
    const float4 v = u[s];
    if ((__float_as_int(v.w) & cell_bits(dx, dy, dz)) != cell_bits(dx, dy, dz)) continue;
#pragma unroll
    for (int k = 0; k < LBE_MAX_SPECIES; ++k)
      if (k < ns) acc[k] += share(ll2f(base + qin[k * N + s]), v.x, v.y, v.z, dx, dy, dz);
  }
#pragma unroll
  for (int k = 0; k < LBE_MAX_SPECIES; ++k)
    if (k < ns) qout[k * N + r] = acc[k] - base;
}

// advect_node for two species (out of line: the rare case of advect_node2)
static __device__ __noinline__ void advect_node2_wide(int N, int r, Offs o, uint32_t m,
                                                      const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                                      int64_t *__restrict__ qout);

// advect_node for two species, each share rounded by acc_round for both
// species at once (no conversion instructions; the same integers as share:
// round-half-even of w tot).  acc_round is exact while |w tot| < 2^43, i.e.
// while the node and its sources hold less than 8 times the bulk amount;
// otherwise (a node near overflow) the node is done again by advect_node.
__device__ __forceinline__ void advect_node2(int N, int r, const Offs &o, uint32_t m,
                                             const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                             int64_t *__restrict__ qout) {
  constexpr float kFast = 8796093022208.f;  // 2^43
  const float4 v0 = u[r];
  const int code0 = __float_as_int(v0.w);
  const long long base = 1LL << kFixBits;
  const long long acc0 = base + qin[r], acc1 = base + qin[N + r];
  const float2 tot = make_float2(ll2f(acc0), ll2f(acc1));
  bool fast = fabsf(tot.x) < kFast && fabsf(tot.y) < kFast;
  unsigned ah0 = 0u, al0 = 0u, ah1 = 0u, al1 = 0u;
  int net = 0;  // acc_round terms added - subtracted
  // outgoing (the share is zero outside the octant of u); shares bound for
  // solid neighbours stay
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(dx, dy, dz)))) continue;
    if ((code0 & cell_bits(dx, dy, dz)) != cell_bits(dx, dy, dz)) continue;
    const float w = ov(dx, v0.x) * ov(dy, v0.y) * ov(dz, v0.z);
    acc_round<-1>(__fmul2_rn(make_float2(w, w), tot), ah0, al0, ah1, al1);
    --net;
  }
  // incoming from every fluid neighbour whose cell reaches r: the source at
  // r - s gives along +s
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13 || !(m & (1u << dir_bit(-dx, -dy, -dz)))) continue;
    const int s = r + o.at(-dx, -dy, -dz);
    const float4 v = u[s];
    if ((__float_as_int(v.w) & cell_bits(dx, dy, dz)) != cell_bits(dx, dy, dz)) continue;
    const float2 ts = make_float2(ll2f(base + qin[s]), ll2f(base + qin[N + s]));
    fast &= fabsf(ts.x) < kFast && fabsf(ts.y) < kFast;
    const float w = ov(dx, v.x) * ov(dy, v.y) * ov(dz, v.z);
    acc_round<1>(__fmul2_rn(make_float2(w, w), ts), ah0, al0, ah1, al1);
    ++net;
  }
  if (fast) {
    qout[r] = acc0 + acc_value(ah0, al0, net) - base;
    qout[N + r] = acc1 + acc_value(ah1, al1, net) - base;
  } else {
    advect_node2_wide(N, r, o, m, qin, u, qout);
  }
}
static __device__ __noinline__ void advect_node2_wide(int N, int r, Offs o, uint32_t m,
                                                      const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                                      int64_t *__restrict__ qout) {
  advect_node(2, N, r, o, m, qin, u, qout);
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

// The potential in fixed point (the FP32 form's master copy): value =
// v 2^-kPhiFixBits.  Its nearest float (ll2f rounds once; the scaling is
// exact).
constexpr float kPhiUnitF = 1.0f / 281474976710656.0f;  // 2^-48
static_assert(kPhiFixBits == 48, "kPhiUnitF is 2^-kPhiFixBits");
__device__ __forceinline__ float fx_to_f(long long v) { return __fmul_rn(ll2f(v), kPhiUnitF); }

// The warm start of extrapolate_node on the fixed-point potential: the same
// polynomials in exact integer arithmetic (no FP64 operation), the float
// copy refreshed, the history (fixed point too) shifted.
__device__ __forceinline__ void extrapolate_fx(long long N, long long i, int64_t *__restrict__ phifx,
                                               int64_t *__restrict__ prev, float *__restrict__ phi32, int history) {
  const long long v = phifx[i], p1 = prev[i];
  if (history > 0) {
    long long e;
    if (history == 1) {
      e = 2 * v - p1;
    } else if (history == 2) {
      e = prev[N + i] + 3 * (v - p1);
    } else {
      const long long p2 = prev[N + i], p3 = prev[2 * N + i];
      e = v + 3 * (v - p1) - 3 * (p1 - p2) + (p2 - p3);
    }
    phifx[i] = e;
    phi32[i] = fx_to_f(e);
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
template <bool ALL>
__device__ __forceinline__ void lap6_ff_(const Offs &o, int r, uint32_t m, const float *__restrict__ hi,
                                         const float *__restrict__ lo, float &S, float &E) {
  const float h0 = hi[r], l0 = lo[r];
  S = 0.f;
  E = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const int j = r + o.at(cx_of(i), cy_of(i), cz_of(i));
    const float w = (float)((c2_of(i) == 1 ? 2 : 1) * ((ALL || (m & (1u << (i - 1)))) ? 1 : 2));
    float d, de;
    two_sum(hi[j], -h0, d, de);  // d + de = hi_j - hi_r exactly
    float t, te;
    two_sum(S, w * d, t, te);  // w is a power of two: w d is exact
    S = t;
    E += te + w * (de + (lo[j] - l0));
  }
}
// (a node whose links all join fluid takes constant weights)
__device__ __forceinline__ void lap6_ff(const Geo &g, int r, int x, int y, int z, uint32_t m,
                                        const float *__restrict__ hi, const float *__restrict__ lo, float &S,
                                        float &E) {
  const Offs o = offsets_of(g, x, y, z);
  if ((m & kLinkBits) == kLinkBits)
    lap6_ff_<true>(o, r, m, hi, lo, S, E);
  else
    lap6_ff_<false>(o, r, m, hi, lo, S, E);
}

// 6 lap_mod(phi)(r) of the fixed-point potential, exactly: the weighted link
// differences (weights 2 axis, 1 diagonal, doubled towards solid) summed in
// 64-bit integers.  |phi| < kPhiMax keeps the sum far below 2^63.
template <bool ALL>
__device__ __forceinline__ long long lap6_fx_(const Offs &o, int r, uint32_t m, const int64_t *__restrict__ v) {
  const long long v0 = v[r];
  const int64_t *__restrict__ vr = v + r;
  long long s = 0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const long long d = vr[o.at(cx_of(i), cy_of(i), cz_of(i))] - v0;
    const int w = (c2_of(i) == 1 ? 2 : 1) * ((ALL || (m & (1u << (i - 1)))) ? 1 : 2);
    s += w == 1 ? d : (w == 2 ? 2 * d : 4 * d);
  }
  return s;
}
__device__ __forceinline__ long long lap6_fx(const Geo &g, int r, int x, int y, int z, uint32_t m,
                                             const int64_t *__restrict__ v) {
  const Offs o = offsets_of(g, x, y, z);
  return (m & kLinkBits) == kLinkBits ? lap6_fx_<true>(o, r, m, v) : lap6_fx_<false>(o, r, m, v);
}
}  // namespace fp32
}  // namespace lbe
