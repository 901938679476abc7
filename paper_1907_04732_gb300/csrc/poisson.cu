// Poisson solve of the LBE step (Sec. "Imposing conducting boundary
// conditions"): find phi on fluid nodes such that
//     lap_mod(phi)(r) + 4 pi l_B rho_el(r) = 0,
// where lap_mod is Eq. DiscreteLaplacianModif (every fluid-solid link
// doubled) and solid nodes hold their electrode potential.  The paper relaxes
// with Eq. SOR and keeps the converged potential; here the same fixed point is
// reached by iterative refinement:
//
//   round:  res = 4 pi l_B rho_el + lap_mod(phi)      (FP64 in the FP64 form;
//           in the FP32 form lap_mod of the fixed-point potential summed
//           exactly in integers, the sum added to the charge term in
//           float-float arithmetic)
//           stop when max_r |res(r)|/diag(r) <= poisson_tol
//           solve A e = res approximately by preconditioned conjugate
//           gradients (FP64 and Jacobi in the FP64 form; FP32 and the
//           multigrid V-cycle of mg.cu in the FP32 form)
//           phi += e                (FP64; FP32 form: e rounded to the
//                                    fixed-point unit, an integer add)
//
// Each step starts from the extrapolation in time of the previous solutions
// (fp32::extrapolate_node, fp32::extrapolate_fx).  The CG is the Chronopoulos-Gear variant: both
// inner products of an iteration come from one reduction phase, so an
// iteration is the vector update (k_cg_a), the preconditioner, and the
// stencil with the dot products (k_cg_b, whose last block runs the scalar
// recurrence).  The whole solve is one CUDA graph: a device-side `while`
// over refinement rounds containing a `while` over CG iterations; kernels set
// the loop conditions, bounded by the round limit and poisson_max_iter.
// Where conditional graph nodes are not available the same kernels run from
// a host loop that polls the device.
//
// Reductions are deterministic: each block reduces in a fixed tree order and
// writes one partial; a single block sums the partials in block order.
#include <stdlib.h>
#include <string.h>

#include "fp32_device.cuh"

namespace lbe {

namespace {

constexpr int kMaxOuter = 24;  // refinement rounds per solve
constexpr int kChunk = 16;     // fallback: iterations between host polls

enum { S_RU = 0, S_WU = 1, S_MAX = 2 };
enum { C_INIT = 0, C_ITER = 1 };

__host__ __device__ constexpr uint32_t nn_bits() {
  uint32_t b = 0;
  for (int i = 1; i < kQ; ++i)
    if (c2_of(i) == 1) b |= 1u << (i - 1);
  return b;
}
constexpr uint32_t kNN = nn_bits();
constexpr uint32_t kNNN = ((1u << 18) - 1) & ~kNN;

// diagonal of -lap_mod at a fluid node: 1/3 per nearest and 1/6 per
// next-nearest link, doubled towards solid (not under the first-order rule,
// kPlainLaplacian); links joining a node to itself (boxes one node wide)
// cancel and are left out.
template <typename T>
__device__ __forceinline__ T diag_t(uint32_t m, uint32_t selfmask) {
  const uint32_t nself = ~selfmask;
  const int dbl = (selfmask & kPlainLaplacian) ? 0 : 1;
  const int nn = __popc(kNN & nself), nns = dbl * __popc(kNN & nself & ~m);
  const int mm = __popc(kNNN & nself), mms = dbl * __popc(kNNN & nself & ~m);
  return (T)(2 * (nn + nns) + (mm + mms)) * (T)(1.0 / 6.0);
}

// lap_mod(v)(r) at a fluid node, FP64.  With the link weights scaled by 6
// (2 nearest, 1 next-nearest, doubled towards solid unless dbl is false:
// the first-order rule) the sum needs one FP64 add per link:
// 6 lap = sum_i w_i v_i - (sum_i w_i) v0, w_i in {1, 2, 4}.
__device__ __forceinline__ double lap_at(const Geo &g, int r, int x, int y, int z, uint32_t m,
                                         const double *__restrict__ v, bool dbl = true) {
  const Offs o = offsets_of(g, x, y, z);
  double s1 = 0.0, s2 = 0.0, s4 = 0.0;
  int wsum = 0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const double vi = v[r + o.at(cx_of(i), cy_of(i), cz_of(i))];
    const int w = (c2_of(i) == 1 ? 2 : 1) * ((m & (1u << (i - 1))) || !dbl ? 1 : 2);
    if (w == 1) s1 += vi;
    else if (w == 2) s2 += vi;
    else s4 += vi;
    wsum += w;
  }
  return (s1 + 2.0 * s2 + 4.0 * s4 - (double)wsum * v[r]) * (1.0 / 6.0);
}

// block-wide sum or max in a fixed order; result valid in thread 0.  The
// FP32 kernels reduce in FP32 within the block (FP64 is slow on this GPU);
// block partials are stored and combined in FP64.
template <bool MAX, typename V = double>
__device__ __forceinline__ V block_reduce(V v) {
  __shared__ V sh[kBlock / 32];
  const int t = flat_tid(), lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const V u = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  V out = 0;
  if (t == 0) {
    out = sh[0];
    for (int w = 1; w < kBlock / 32; ++w) out = MAX ? fmax(out, sh[w]) : out + sh[w];
  }
  return out;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, unsigned v) {
  if (use) cudaGraphSetConditional(h, v);
}

// Last-block-done: after a block has written its partials it takes a ticket;
// the block that takes the last ticket sees every partial (each block fenced
// its writes before its ticket) and finishes the reduction.  No block waits.
__device__ __forceinline__ bool last_block(PoissonCtl *c, int nblk) {
  __shared__ int last;
  __syncthreads();
  if (flat_tid() == 0) {
    __threadfence();
    last = atomicAdd(&c->arrive, 1) == nblk - 1;
  }
  __syncthreads();
  return last;
}

// two sums and a max over the block in one pass (the order of block_reduce
// for each value, with one pair of barriers); results valid in thread 0
__device__ __forceinline__ void block_reduce3(double &a, double &b, double &m) {
  __shared__ double sh[3][kBlock / 32];
  const int t = flat_tid(), lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ua = __shfl_down_sync(0xffffffffu, a, o), ub = __shfl_down_sync(0xffffffffu, b, o),
                 um = __shfl_down_sync(0xffffffffu, m, o);
    a += ua;
    b += ub;
    m = fmax(m, um);
  }
  __syncthreads();
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
    sh[2][wid] = m;
  }
  __syncthreads();
  if (t == 0) {
    a = sh[0][0];
    b = sh[1][0];
    m = sh[2][0];
    for (int w = 1; w < kBlock / 32; ++w) {
      a += sh[0][w];
      b += sh[1][w];
      m = fmax(m, sh[2][w]);
    }
  }
}

// sums/max of the partials in block order (every thread of the block calls).
// All of a thread's partials are loaded before any is added (one L2 latency
// instead of one per stride of the block), then summed in the same order.
__device__ __forceinline__ void reduce_partials(const double *part, int nblk, double *ru, double *wu, double *mx) {
  constexpr int kPer = (kSolveBlocks + kBlock - 1) / kBlock;  // the solve launches at most kSolveBlocks blocks
  double pa[kPer], pb[kPer], pm[kPer];
  const int t = flat_tid();
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = t + k * kBlock;
    const bool in = i < nblk;
    pa[k] = in ? __ldcg(part + S_RU * nblk + i) : 0.0;
    pb[k] = in ? __ldcg(part + S_WU * nblk + i) : 0.0;
    pm[k] = in ? __ldcg(part + S_MAX * nblk + i) : 0.0;
  }
  double a = 0.0, b = 0.0, m = 0.0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (t + k * kBlock < nblk) {
      a += pa[k];
      b += pb[k];
      m = fmax(m, pm[k]);
    }
  }
  for (int i = t + kPer * kBlock; i < nblk; i += kBlock) {  // a larger launch (not used by the solve)
    a += __ldcg(part + S_RU * nblk + i);
    b += __ldcg(part + S_WU * nblk + i);
    m = fmax(m, __ldcg(part + S_MAX * nblk + i));
  }
  block_reduce3(a, b, m);
  *ru = a;
  *wu = b;
  *mx = m;
}

// outer test of a refinement round (thread 0 of the last block of k_res):
// converged, out of rounds or out of iterations?  A round that did not
// halve the residual means the tolerance lies below what the arithmetic
// resolves: the solve stops there (LBE_ERR_NOCONVERGE) instead of repeating
// rounds that cannot help.
__device__ void outer_check(PoissonCtl *c, double m, double tol, int maxit, cudaGraphConditionalHandle hout,
                            cudaGraphConditionalHandle hin, int use_cond, int set_hin) {
  const double prev = c->res;
  c->res = m;
  int done = 0;
  if (m <= tol) {
    done = 1;
  } else if (!(m == m) || m > 1e300) {
    done = 1;
    c->status = LBE_ERR_NONFINITE;
  } else if (c->rounds >= kMaxOuter || c->solve_iters >= maxit || (c->rounds >= 1 && m > 0.5 * prev)) {
    done = 1;
    c->status = LBE_ERR_NOCONVERGE;
  }
  c->outer_done = done;
  c->inner_done = done;  // nothing more of the round runs once converged
  c->rounds += 1;
  c->total_rounds += 1;
  set_cond(hout, use_cond, done ? 0u : 1u);
  if (done && set_hin) set_cond(hin, use_cond, 0u);
}

// scalar recurrence of the Chronopoulos-Gear CG and the inner stopping test
// (relative reduction eta of the round's starting residual); thread 0 of the
// last block of k_cg_b
__device__ void cg_scalars(PoissonCtl *c, double gam, double del, double mx, double eta, double tol_abs, int maxit,
                           int mode, cudaGraphConditionalHandle hin, int use_cond) {
  int done = 0;
  if (mode == C_INIT) {
    c->res0 = c->res;
    c->beta = 0.0;
    c->alpha = gam / del;
    c->gamma = gam;
    if (!(del > 0.0) || !(gam > 0.0)) done = 1;  // zero residual: nothing to solve
  } else {
    c->solve_iters += 1;
    c->total_iters += 1;
    if (mx <= fmax(eta * c->res0, tol_abs)) {
      done = 1;
    } else if (!(mx == mx) || mx > 1e300 || !(del == del)) {
      done = 1;
      c->status = LBE_ERR_NONFINITE;
      c->outer_done = 1;
    } else if (c->solve_iters >= maxit) {
      done = 1;
    } else {
      const double beta = gam / c->gamma;
      const double den = del - beta * gam / c->alpha;
      if (!(den > 0.0) || !(gam > 0.0)) {
        done = 1;  // breakdown: the correction is converged to rounding
      } else {
        c->beta = beta;
        c->alpha = gam / den;
        c->gamma = gam;
      }
    }
  }
  c->inner_done = done;
  set_cond(hin, use_cond, done ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// start of a solve: fold the previous solve into the sticky fields, reset
__global__ void k_solve_reset(PoissonCtl *c) {
  if (c->status && !c->sticky_status) c->sticky_status = c->status;
  if (c->solve_iters > c->max_solve_iters) c->max_solve_iters = c->solve_iters;
  c->outer_done = 0;
  c->inner_done = 0;
  c->rounds = 0;
  c->status = 0;
  c->solve_iters = 0;
  c->solves += 1;
}

// Residual of the current potential; seeds the inner solve:
// r = (T)res, u = r/diag, x = p = s = 0.  Partial max |res|/diag.
// MODE: R_N64 the FP64 form (FP64 potential and n); R_FX the FP32 form for
// a 1:1 salt: the fixed-point potential's Laplacian summed exactly in
// integers, the charge term from the fixed-point solute, both combined in
// float-float arithmetic; R_FXG the FP32 form for other salts (the exact
// Laplacian and the charge density in FP64); R_RHS a given rhs (linear
// solve A x = rhs with an FP64 iterate; its relative test also needs
// max |rhs|/diag, kept in the otherwise idle (r,u) partial slots); R_RHS_FF
// the same in float-float arithmetic (rhs values that are floats, x held as
// two floats).
enum { R_N64 = 0, R_FXG = 1, R_RHS = 2, R_FX = 3, R_RHS_FF = 4 };
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock) k_res(const Geo g, int zpt, const Phys P, const P32 P3,
                                                const uint32_t *__restrict__ mask, const double *__restrict__ n64,
                                                const int64_t *__restrict__ nq, const double *__restrict__ rhs,
                                                const double *__restrict__ phi, const float *__restrict__ phi_hi,
                                                const float *__restrict__ phi_lo, const int64_t *__restrict__ phifx,
                                                float c6_hi, float c6_lo,
                                                T *__restrict__ r,
                                                T *__restrict__ u, T *__restrict__ x, T *__restrict__ p,
                                                T *__restrict__ s, double *__restrict__ part, int nblk,
                                                PoissonCtl *c, double tol, double tol_rel, int maxit,
                                                cudaGraphConditionalHandle hout, cudaGraphConditionalHandle hin,
                                                int use_cond, int set_hin) {
  constexpr bool RHS = MODE == R_RHS || MODE == R_RHS_FF;
  float mx = 0.f, mb = 0.f;
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    const uint32_t m = mask[i];
    if (!(m & kFluidBit)) {
      r[i] = u[i] = x[i] = p[i] = s[i] = (T)0;
      continue;
    }
    if (MODE == R_FX) {
      // 6 res = 6 lap + 6 (4 pi l_B s) (q+ - q-): 6 lap exact in fixed
      // point, split into float-float (the nearest float of the integer sum
      // and the float of its exact remainder), the charge term in
      // float-float too
      const long long L6 = fp32::lap6_fx(g, (int)i, X, Y, Z, m, phifx);
      const float Lh = fp32::ll2f(L6);
      const float Ll = fp32::ll2f(L6 - fp32::f2ll_rn(Lh));
      const float S = __fmul_rn(Lh, fp32::kPhiUnitF), E = __fmul_rn(Ll, fp32::kPhiUnitF);
      const long long dq = nq[i] - nq[g.N + i];
      const float dq_hi = fp32::ll2f(dq);
      const float dq_lo = fp32::ll2f(dq - fp32::f2ll_rn(dq_hi));  // exact remainder
      const float B = c6_hi * dq_hi;
      const float Be = fmaf(c6_hi, dq_hi, -B) + (c6_hi * dq_lo + c6_lo * dq_hi);  // product error and tails
      float t, te;
      fp32::two_sum(S, B, t, te);
      const float rt = (t + (te + (E + Be))) * (1.f / 6.f);
      const float dinv = 1.f / diag_t<float>(m, P.selfmask);
      r[i] = (T)rt;
      u[i] = (T)(rt * dinv);
      x[i] = p[i] = s[i] = (T)0;
      mx = fmaxf(mx, finite_or_inf(fabsf(rt) * dinv));
      continue;
    }
    if (MODE == R_RHS_FF) {
      // 6 res = 6 rhs + 6 lap(x), x = hi + lo, in float-float; rhs is a float
      float S, E;
      fp32::lap6_ff(g, (int)i, X, Y, Z, m, phi_hi, phi_lo, S, E);
      const float bf = (float)rhs[i];
      const float B = 6.f * bf, Be = fmaf(6.f, bf, -B);  // 6 rhs = B + Be exactly
      float t, te;
      fp32::two_sum(S, B, t, te);
      const float rt = (t + (te + (E + Be))) * (1.f / 6.f);
      const float dinv = 1.f / diag_t<float>(m, P.selfmask);
      r[i] = (T)rt;
      u[i] = (T)(rt * dinv);
      x[i] = p[i] = s[i] = (T)0;
      mx = fmaxf(mx, finite_or_inf(fabsf(rt) * dinv));
      mb = fmaxf(mb, finite_or_inf(fabsf(bf) * dinv));
      continue;
    }
    double b;
    if (MODE == R_RHS) {
      b = rhs[i];
    } else {
      double q = 0.0;
      for (int k = 0; k < P.ns; ++k)
        q += P.z[k] * (MODE == R_FXG ? P3.rbd[k] + P3.sd[k] * (double)nq[k * g.N + i] : n64[k * g.N + i]);
      b = P.four_pi_lb * q;
    }
    const double lap = MODE == R_FXG
                           ? (double)fp32::lap6_fx(g, (int)i, X, Y, Z, m, phifx) * (1.0 / 281474976710656.0 / 6.0)
                           : lap_at(g, (int)i, X, Y, Z, m, phi, !(P.selfmask & kPlainLaplacian));
    const double rr = b + lap;
    const T rt = (T)rr;
    const T dinv = (T)1 / diag_t<T>(m, P.selfmask);
    r[i] = rt;
    u[i] = rt * dinv;
    x[i] = p[i] = s[i] = (T)0;
    mx = fmaxf(mx, finite_or_inf(fabsf((float)rr) * (float)dinv));  // the stopping test needs no FP64
    if (MODE == R_RHS) mb = fmaxf(mb, finite_or_inf(fabsf((float)b) * (float)dinv));
  }
  mx = block_reduce<true, float>(mx);
  if (flat_tid() == 0) part[S_MAX * nblk + flat_bid()] = (double)mx;
  if (RHS) {
    mb = block_reduce<true, float>(mb);
    if (flat_tid() == 0) part[S_RU * nblk + flat_bid()] = (double)mb;
  }
  if (!last_block(c, nblk)) return;
  double m = 0.0, ref = 0.0;
  for (int i = flat_tid(); i < nblk; i += kBlock) {
    m = fmax(m, __ldcg(part + S_MAX * nblk + i));
    if (RHS) ref = fmax(ref, __ldcg(part + S_RU * nblk + i));
  }
  m = block_reduce<true>(m);
  if (RHS) ref = block_reduce<true>(ref);
  if (flat_tid() == 0) {
    c->arrive = 0;
    if (RHS) c->ref = ref;
    outer_check(c, m, RHS ? fmax(tol, tol_rel * ref) : tol, maxit, hout, hin, use_cond, set_hin);
  }
}

// stencil + dot products: w = A u; partials (r,u), (w,u); the last block
// runs the scalar recurrence
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_b(const Geo g, int zpt, uint32_t selfmask,
                                                 const uint32_t *__restrict__ mask, const T *__restrict__ u,
                                                 const T *__restrict__ r, T *__restrict__ w,
                                                 double *__restrict__ part, int nblk, PoissonCtl *c, double eta,
                                                 double tol_abs, int maxit, int mode,
                                                 cudaGraphConditionalHandle hin, int use_cond) {
  if (c->inner_done) return;
  T ru = 0, wu = 0;
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    const uint32_t m = mask[i];
    if (!(m & kFluidBit)) continue;
    const T u0 = u[i];
    const Offs o = offsets_of(g, X, Y, Z);
    const T *__restrict__ ui = u + i;
    T sum = 0;
    if (all_links(m, selfmask)) {  // the same sum without the weight tests
#pragma unroll
      for (int l = 1; l < kQ; ++l) sum += (T)lapc_of(l) * ui[o.at(cx_of(l), cy_of(l), cz_of(l))];
    } else {
#pragma unroll
      for (int l = 1; l < kQ; ++l) {  // every neighbour read; a zero weight drops it
        const uint32_t b = 1u << (l - 1);
        const T ul = ui[o.at(cx_of(l), cy_of(l), cz_of(l))];
        sum += ((selfmask & b) || !(m & b) ? (T)0 : (T)lapc_of(l)) * ul;
      }
    }
    const T wv = diag_t<T>(m, selfmask) * u0 - sum;
    w[i] = wv;
    ru += r[i] * u0;
    wu += wv * u0;
  }
  const T a = block_reduce<false, T>(ru);
  const T b = block_reduce<false, T>(wu);
  if (flat_tid() == 0) {
    part[S_RU * nblk + flat_bid()] = (double)a;
    part[S_WU * nblk + flat_bid()] = (double)b;
  }
  if (!last_block(c, nblk)) return;
  double gam, del, mx;
  reduce_partials(part, nblk, &gam, &del, &mx);
  if (flat_tid() == 0) {
    c->arrive = 0;
    cg_scalars(c, gam, del, mx, eta, tol_abs, maxit, mode, hin, use_cond);
  }
}

// vector update: p = u + beta p, s = w + beta s, x += alpha p,
// r -= alpha s, u = r/diag; partial max |r|/diag
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_a(const Geo g, int zpt, uint32_t selfmask,
                                                 const uint32_t *__restrict__ mask, T *__restrict__ x,
                                                 T *__restrict__ r, T *__restrict__ u, const T *__restrict__ w,
                                                 T *__restrict__ p, T *__restrict__ s, double *__restrict__ part,
                                                 int nblk, const PoissonCtl *c) {
  if (c->inner_done) return;
  const T alpha = (T)c->alpha, beta = (T)c->beta;
  T mx = 0;
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    const uint32_t m = mask[i];
    if (!(m & kFluidBit)) continue;
    const T pv = u[i] + beta * p[i];
    const T sv = w[i] + beta * s[i];
    p[i] = pv;
    s[i] = sv;
    x[i] += alpha * pv;
    const T rv = r[i] - alpha * sv;
    r[i] = rv;
    const T dinv = (T)1 / diag_t<T>(m, selfmask);
    u[i] = rv * dinv;
    mx = fmax(mx, finite_or_inf(fabs(rv) * dinv));
  }
  const T v = block_reduce<true, T>(mx);
  if (flat_tid() == 0) part[S_MAX * nblk + flat_bid()] = (double)v;
}

// warm start of a step's solve on fluid nodes (fp32::extrapolate_node); the
// FP32 form with flow does this inside the advection kernel instead
__global__ void k_extrapolate(const Geo g, int zpt, const uint32_t *__restrict__ mask, double *__restrict__ phi,
                              double *__restrict__ prev, float *__restrict__ phi32, float *__restrict__ phi_lo,
                              int history) {
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    if (mask[i] & kFluidBit) fp32::extrapolate_node(g.N, i, phi, prev, phi32, phi_lo, history);
  }
}

// FP32 form: the fixed-point potential += e (rounded to the fixed-point
// unit) on fluid nodes and its float copy; |phi| reaching kPhiMax raises
// range flag 4
__global__ void k_correct_fx(const Geo g, int zpt, const uint32_t *__restrict__ mask, const float *__restrict__ e,
                             int64_t *__restrict__ phifx, float *__restrict__ phi32, int *__restrict__ flag) {
  constexpr float kMaxFx = (float)(kPhiMax * 281474976710656.0);  // kPhiMax 2^kPhiFixBits
  bool over = false;
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    if (!(mask[i] & kFluidBit)) continue;
    const float d = __fmul_rn(e[i], 281474976710656.0f);  // e 2^kPhiFixBits, exact
    if (!(fabsf(d) < kMaxFx)) {  // also NaN
      over = true;
      continue;
    }
    const long long v = phifx[i] + fp32::f2ll_rn(d);
    over |= !(fabsf(fp32::ll2f(v)) < kMaxFx);
    phifx[i] = v;
    phi32[i] = fp32::fx_to_f(v);
  }
  if (over) atomicOr(flag, 4);
}

// FP32 form without flow (no advection kernel to carry it): the warm start
// on the fixed-point potential
__global__ void k_extrapolate_fx(const Geo g, int zpt, const uint32_t *__restrict__ mask, int64_t *__restrict__ phifx,
                                 int64_t *__restrict__ prev, float *__restrict__ phi32, int history) {
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    if (mask[i] & kFluidBit) fp32::extrapolate_fx(g.N, i, phifx, prev, phi32, history);
  }
}

// phi64 += e on fluid nodes; with phi32 given its float split follows
// (the FP64 form, and the linear solves' FP64 iterates)
template <typename T>
__global__ void k_correct(const Geo g, int zpt, const uint32_t *__restrict__ mask, const T *__restrict__ e,
                          double *__restrict__ phi, float *__restrict__ phi32, float *__restrict__ phi_lo) {
  for (int kz = 0; kz < zpt; ++kz) {
    int X, Y, Z;
    long long i;
    if (!node_of(g, zpt, kz, X, Y, Z, i)) continue;
    double v = phi[i];
    if (e && (mask[i] & kFluidBit)) {
      v += (double)e[i];
      phi[i] = v;
    }
    if (phi32) {
      const float hi = (float)v;
      phi32[i] = hi;
      if (phi_lo) phi_lo[i] = (float)(v - (double)hi);
    }
  }
}

// ---------------------------------------------------------------------------
// kernel argument storage for graph nodes (values are copied at node creation)
struct Args {
  Geo g;
  int zpt, nblk, maxit, use_cond = 1, mode_init = C_INIT, mode_iter = C_ITER, hin_no = 0, hin_yes = 1;
  Phys P;
  P32 P3;
  uint32_t selfmask;
  double tol, tol_rel = 0.0, eta, tol_inner;
  const uint32_t *mask;
  const double *n64;
  const int64_t *nq;
  const double *rhs = nullptr;
  double *phi;
  float *phi32, *phi_lo = nullptr;
  float c6_hi = 0.f, c6_lo = 0.f;  // 6 * 4 pi l_B * s, as two floats (R_FX)
  int64_t *phifx = nullptr;        // the FP32 form's fixed-point potential
  int *flag = nullptr;             // the FP32 form's range flags
  void *r, *u, *w, *x, *p, *s;
  double *part;
  PoissonCtl *c;
  cudaGraphConditionalHandle hout = 0, hin = 0;
};

cudaError_t add_kernel(cudaGraph_t gr, cudaGraphNode_t *last, void *func, dim3 grid, dim3 block, void **args) {
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = func;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.kernelParams = args;
  cudaGraphNode_t n;
  cudaError_t e = cudaGraphAddKernelNode(&n, gr, *last ? last : nullptr, *last ? 1 : 0, &kp);
  if (e == cudaSuccess) *last = n;
  return e;
}

cudaError_t add_while(cudaGraph_t gr, cudaGraphNode_t *last, cudaGraphConditionalHandle h, cudaGraph_t *body) {
  // cudaGraphNodeParams has no default constructor: zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams *np = reinterpret_cast<cudaGraphNodeParams *>(raw);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t n;
  cudaError_t e = cudaGraphAddNode(&n, gr, *last ? last : nullptr, nullptr, *last ? 1 : 0, np);
  if (e == cudaSuccess) {
    *last = n;
    *body = np->conditional.phGraph_out[0];
  }
  return e;
}

template <typename T>
void fill_args(lbe_handle *h, Args &A) {
  PoissonWork &w = h->pw;
  const long long N = h->geo.N;
  T *base = (T *)w.vec;
  A.g = h->geo;
  A.zpt = w.L.zpt;
  A.nblk = (int)w.L.nblk();
  A.maxit = h->prm.poisson_max_iter;
  A.P = h->phys;
  A.P3 = h->p32;
  A.selfmask = h->phys.selfmask;
  A.tol = h->prm.poisson_tol;
  A.eta = sizeof(T) == 4 ? 1e-4 : 1e-9;
  // an inner solve need not go below a fraction of the outer tolerance:
  // 0.8 measured 2.15 CG iterations per step on the 64x64x256
  // electro-osmosis lattice against 2.9 at 0.25 and 2.4 at 0.5, with no
  // extra refinement round (the outer test still decides convergence)
  A.tol_inner = 0.8 * A.tol;
  A.mask = h->mask;
  A.n64 = h->n;
  A.nq = h->q;
  A.phi = h->phi;
  A.phi32 = h->phi32;
  A.phifx = h->phifx;
  A.flag = h->flag;
  {
    const double c6 = 6.0 * h->phys.four_pi_lb * h->p32.sd[0];
    A.c6_hi = (float)c6;
    A.c6_lo = (float)(c6 - (double)A.c6_hi);
  }
  A.r = base;
  A.u = base + N;
  A.w = base + 2 * N;
  A.x = base + 3 * N;
  A.p = base + 4 * N;
  A.s = base + 5 * N;
  A.part = w.partial;
  A.c = w.ctl;
}

template <typename T>
cudaError_t build_graph(lbe_handle *h, Args &A, cudaGraphExec_t *exec) {
  const Launch &L = h->pw.L;
  const dim3 one(1);
  const bool fixed = h->prm.precision == LBE_FP32;
  void *f_res = A.rhs ? (A.phi32 && A.phi_lo ? (void *)k_res<T, R_RHS_FF> : (void *)k_res<T, R_RHS>)
                      : (fixed ? (h->p32.salt11 ? (void *)k_res<T, R_FX> : (void *)k_res<T, R_FXG>)
                               : (void *)k_res<T, R_N64>);
  // the FP32 form's own solve corrects its fixed-point potential; the FP64
  // form and the linear solves correct an FP64 iterate
  const bool corr_fx = fixed && !A.rhs;
  cudaGraph_t G = nullptr;
  cudaError_t e = cudaGraphCreate(&G, 0);
  if (e != cudaSuccess) return e;
  cudaGraphNode_t last = nullptr, lo = nullptr, li = nullptr;
  cudaGraph_t body_out = nullptr, body_in = nullptr;
  void *a_reset[] = {&A.c};
  // the residual before the round loop must not touch the inner loop's
  // condition (it belongs to the loop body); the one closing a round does
  void *a_res0[] = {&A.g,     &A.zpt,   &A.P,      &A.P3,    &A.mask,    &A.n64,   &A.nq, &A.rhs,
                    &A.phi,   &A.phi32, &A.phi_lo, &A.phifx, &A.c6_hi,   &A.c6_lo, &A.r,  &A.u,
                    &A.x,     &A.p,     &A.s,      &A.part,  &A.nblk,    &A.c,     &A.tol, &A.tol_rel,
                    &A.maxit, &A.hout,  &A.hin,    &A.use_cond, &A.hin_no};
  void *a_res[] = {&A.g,     &A.zpt,   &A.P,      &A.P3,    &A.mask,    &A.n64,   &A.nq, &A.rhs,
                   &A.phi,   &A.phi32, &A.phi_lo, &A.phifx, &A.c6_hi,   &A.c6_lo, &A.r,  &A.u,
                   &A.x,     &A.p,     &A.s,      &A.part,  &A.nblk,    &A.c,     &A.tol, &A.tol_rel,
                   &A.maxit, &A.hout,  &A.hin,    &A.use_cond, &A.hin_yes};
  void *a_bi[] = {&A.g, &A.zpt, &A.selfmask, &A.mask, &A.u, &A.r, &A.w, &A.part, &A.nblk, &A.c,
                  &A.eta, &A.tol_inner, &A.maxit, &A.mode_init, &A.hin, &A.use_cond};
  void *a_bt[] = {&A.g, &A.zpt, &A.selfmask, &A.mask, &A.u, &A.r, &A.w, &A.part, &A.nblk, &A.c,
                  &A.eta, &A.tol_inner, &A.maxit, &A.mode_iter, &A.hin, &A.use_cond};
  void *a_a[] = {&A.g, &A.zpt, &A.selfmask, &A.mask, &A.x, &A.r, &A.u, &A.w, &A.p, &A.s, &A.part, &A.nblk, &A.c};
  void *a_cor[] = {&A.g, &A.zpt, &A.mask, &A.x, &A.phi, &A.phi32, &A.phi_lo};
  void *a_corfx[] = {&A.g, &A.zpt, &A.mask, &A.x, &A.phifx, &A.phi32, &A.flag};
  // reset -> residual test -> while (not converged) { V-cycle -> CG -> correct
  // -> residual test }: a converged test ends the solve without running the
  // rest of a round
  e = cudaGraphConditionalHandleCreate(&A.hout, G, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = add_kernel(G, &last, (void *)k_solve_reset, one, one, a_reset);
  if (e == cudaSuccess) e = add_kernel(G, &last, f_res, L.grid, L.block, a_res0);
  if (e == cudaSuccess) e = add_while(G, &last, A.hout, &body_out);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&A.hin, body_out, 0, 0);
  const bool mg = sizeof(T) == 4 && h->mg.nlev >= 2;
  if (e == cudaSuccess && mg) e = mg_vcycle(h, (const float *)A.r, (float *)A.u, A.c, body_out, &lo, nullptr);
  if (e == cudaSuccess) e = add_kernel(body_out, &lo, (void *)k_cg_b<T>, L.grid, L.block, a_bi);
  if (e == cudaSuccess) e = add_while(body_out, &lo, A.hin, &body_in);
  if (e == cudaSuccess) e = add_kernel(body_in, &li, (void *)k_cg_a<T>, L.grid, L.block, a_a);
  if (e == cudaSuccess && mg) e = mg_vcycle(h, (const float *)A.r, (float *)A.u, A.c, body_in, &li, nullptr);
  if (e == cudaSuccess) e = add_kernel(body_in, &li, (void *)k_cg_b<T>, L.grid, L.block, a_bt);
  if (e == cudaSuccess)
    e = corr_fx ? add_kernel(body_out, &lo, (void *)k_correct_fx, L.grid, L.block, a_corfx)
                : add_kernel(body_out, &lo, (void *)k_correct<T>, L.grid, L.block, a_cor);
  if (e == cudaSuccess) e = add_kernel(body_out, &lo, f_res, L.grid, L.block, a_res);
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, G, 0);
  cudaGraphDestroy(G);
  return e;
}

// host-driven fallback: the same kernels, polling the control block
template <typename T>
int solve_polled(lbe_handle *h, Args &A) {
  PoissonWork &w = h->pw;
  const Launch &L = w.L;
  cudaStream_t st = h->stream;
  const bool fixed = h->prm.precision == LBE_FP32;
  A.use_cond = 0;
  k_solve_reset<<<1, 1, 0, st>>>(A.c);
  h->launches += 1;
  for (int round = 0; round <= kMaxOuter; ++round) {
    {
      auto kres = A.rhs ? (A.phi32 && A.phi_lo ? k_res<T, R_RHS_FF> : k_res<T, R_RHS>)
                        : (fixed ? (h->p32.salt11 ? k_res<T, R_FX> : k_res<T, R_FXG>) : k_res<T, R_N64>);
      kres<<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.P, A.P3, A.mask, A.n64, A.nq, A.rhs, A.phi, A.phi32, A.phi_lo,
                                        A.phifx, A.c6_hi, A.c6_lo, (T *)A.r, (T *)A.u, (T *)A.x, (T *)A.p,
                                        (T *)A.s, A.part, A.nblk, A.c, A.tol, A.tol_rel, A.maxit, 0, 0, 0, 0);
    }
    const bool mg = sizeof(T) == 4 && h->mg.nlev >= 2;
    if (mg && mg_vcycle(h, (const float *)A.r, (float *)A.u, A.c, nullptr, nullptr, st) != cudaSuccess)
      return LBE_ERR_CUDA;
    k_cg_b<T><<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.selfmask, A.mask, (T *)A.u, (T *)A.r, (T *)A.w, A.part,
                                           A.nblk, A.c, A.eta, A.tol_inner, A.maxit, C_INIT, 0, 0);
    h->launches += 2;
    const long long max_chunks = (long long)A.maxit / kChunk + 2;
    for (long long ch = 0;; ++ch) {
      cudaError_t e = cudaMemcpyAsync(w.ctl_host, w.ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        h->err = std::string("poisson: ") + cudaGetErrorString(e);
        return LBE_ERR_CUDA;
      }
      if (w.ctl_host->inner_done || ch >= max_chunks) break;
      for (int k = 0; k < kChunk; ++k) {
        k_cg_a<T><<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.selfmask, A.mask, (T *)A.x, (T *)A.r, (T *)A.u,
                                               (T *)A.w, (T *)A.p, (T *)A.s, A.part, A.nblk, A.c);
        if (mg && mg_vcycle(h, (const float *)A.r, (float *)A.u, A.c, nullptr, nullptr, st) != cudaSuccess)
          return LBE_ERR_CUDA;
        k_cg_b<T><<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.selfmask, A.mask, (T *)A.u, (T *)A.r, (T *)A.w,
                                               A.part, A.nblk, A.c, A.eta, A.tol_inner, A.maxit, C_ITER, 0, 0);
      }
      h->launches += 2 * kChunk;
    }
    if (fixed && !A.rhs)
      k_correct_fx<<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.mask, (const float *)A.x, A.phifx, A.phi32, A.flag);
    else
      k_correct<T><<<L.grid, L.block, 0, st>>>(A.g, A.zpt, A.mask, (const T *)A.x, A.phi, A.phi32, A.phi_lo);
    h->launches += 1;
    if (w.ctl_host->outer_done) break;
  }
  return cudaGetLastError() == cudaSuccess ? LBE_OK : LBE_ERR_CUDA;
}

template <typename T>
int solve_t(lbe_handle *h) {
  PoissonWork &w = h->pw;
  // one graph per solute buffer (flow-off steps swap the two buffers)
  const void *key = h->prm.precision == LBE_FP32 ? (const void *)h->q : (const void *)h->n;
  int slot = -1;
  for (int k = 0; k < 2; ++k)
    if (w.exec[k] && w.exec_key[k] == key) slot = k;
  if (slot < 0 && w.graph_ok) {
    slot = !w.exec[0] ? 0 : (!w.exec[1] ? 1 : 0);
    if (w.exec[slot]) cudaGraphExecDestroy(w.exec[slot]);
    w.exec[slot] = nullptr;
    Args A;
    fill_args<T>(h, A);
    cudaError_t e = build_graph<T>(h, A, &w.exec[slot]);
    if (e != cudaSuccess) {
      cudaGetLastError();  // clear the error; use the polled loop from now on
      w.graph_ok = false;
      w.exec[slot] = nullptr;
      slot = -1;
    } else {
      w.exec_key[slot] = key;
    }
  }
  if (slot >= 0) {
    cudaError_t e = cudaGraphLaunch(w.exec[slot], h->stream);
    if (e != cudaSuccess) {
      h->err = std::string("poisson graph launch: ") + cudaGetErrorString(e);
      return LBE_ERR_CUDA;
    }
    return LBE_OK;
  }
  Args A;
  fill_args<T>(h, A);
  return solve_polled<T>(h, A);
}

}  // namespace

cudaError_t poisson_alloc(lbe_handle *h) {
  PoissonWork &w = h->pw;
  const long long N = h->geo.N;
  w.L = make_launch(h->geo, kSolveBlocks);
  const size_t tsz = h->prm.precision == LBE_FP32 ? sizeof(float) : sizeof(double);
  cudaError_t e;
  if ((e = cudaMalloc(&w.vec, tsz * 6 * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.partial, sizeof(double) * 3 * w.L.nblk())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.phi_prev, sizeof(double) * kHist * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.ctl, sizeof(PoissonCtl))) != cudaSuccess) return e;
  if ((e = cudaMemset(w.ctl, 0, sizeof(PoissonCtl))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&w.ctl_host, sizeof(PoissonCtl))) != cudaSuccess) return e;
  // LBE_POISSON_GRAPH=0 runs the solves from the host loop (same kernels),
  // e.g. for profilers that do not follow conditional graph nodes
  const char *env = getenv("LBE_POISSON_GRAPH");
  w.graph_ok = !(env && env[0] == '0');
  return cudaSuccess;
}

void poisson_free(lbe_handle *h) {
  PoissonWork &w = h->pw;
  for (int k = 0; k < 2; ++k)
    if (w.exec[k]) cudaGraphExecDestroy(w.exec[k]);
  if (w.exec_lin) cudaGraphExecDestroy(w.exec_lin);
  cudaFree(w.vec);
  cudaFree(w.partial);
  cudaFree(w.phi_prev);
  cudaFree(w.ctl);
  if (w.ctl_host) cudaFreeHost(w.ctl_host);
  w = PoissonWork{};
}

void poisson_drop_graphs(lbe_handle *h) {
  PoissonWork &w = h->pw;
  for (int k = 0; k < 2; ++k) {
    if (w.exec[k]) cudaGraphExecDestroy(w.exec[k]);
    w.exec[k] = nullptr;
    w.exec_key[k] = nullptr;
  }
  if (w.exec_lin) cudaGraphExecDestroy(w.exec_lin);
  w.exec_lin = nullptr;
  w.lin_key[0] = w.lin_key[1] = w.lin_key[2] = nullptr;
}

int poisson_solve_linear(lbe_handle *h, const double *rhs, double *x, double tol_abs, double tol_rel, float *x_hi,
                         float *x_lo) {
  if (h->prm.precision != LBE_FP32) {
    h->err = "linear solve: FP32 form only";
    return LBE_ERR_STATE;
  }
  PoissonWork &w = h->pw;
  Args A;
  fill_args<float>(h, A);
  A.rhs = rhs;
  A.phi = x;
  A.phi32 = x_hi;
  A.phi_lo = x_lo;
  if (x_hi && x_lo) {  // the split of the starting x; the corrections keep it current
    k_correct<float><<<w.L.grid, w.L.block, 0, h->stream>>>(h->geo, w.L.zpt, h->mask, nullptr, x, x_hi, x_lo);
    if (cudaGetLastError() != cudaSuccess) return LBE_ERR_CUDA;
  }
  A.tol = tol_abs;
  A.tol_rel = tol_rel;
  A.tol_inner = 0.25 * tol_abs;
  if (!w.graph_ok) return solve_polled<float>(h, A);
  if (!w.exec_lin || w.lin_key[0] != rhs || w.lin_key[1] != x || w.lin_key[2] != x_hi) {
    if (w.exec_lin) cudaGraphExecDestroy(w.exec_lin);
    w.exec_lin = nullptr;
    cudaError_t e = build_graph<float>(h, A, &w.exec_lin);
    if (e != cudaSuccess) {
      h->err = std::string("linear solve graph: ") + cudaGetErrorString(e);
      w.exec_lin = nullptr;
      return LBE_ERR_CUDA;
    }
    w.lin_key[0] = rhs;
    w.lin_key[1] = x;
    w.lin_key[2] = x_hi;
  }
  cudaError_t e = cudaGraphLaunch(w.exec_lin, h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("linear solve graph launch: ") + cudaGetErrorString(e);
    return LBE_ERR_CUDA;
  }
  return LBE_OK;
}

int poisson_enqueue(lbe_handle *h, bool extrapolate, bool extrapolated) {
  PoissonWork &w = h->pw;
  if (extrapolate) {
    if (!extrapolated) {
      if (h->prm.precision == LBE_FP32)
        k_extrapolate_fx<<<w.L.grid, w.L.block, 0, h->stream>>>(h->geo, w.L.zpt, h->mask, h->phifx,
                                                                (int64_t *)w.phi_prev, h->phi32, w.history);
      else
        k_extrapolate<<<w.L.grid, w.L.block, 0, h->stream>>>(h->geo, w.L.zpt, h->mask, h->phi, w.phi_prev, nullptr,
                                                           nullptr, w.history);
      h->launches += 1;
    }
    if (w.history < kHist) w.history += 1;
  } else {
    w.history = 0;
  }
  if (h->prm.precision == LBE_FP32) {
    h->phi64_stale = true;  // the solve moves the fixed-point potential
    return solve_t<float>(h);
  }
  return solve_t<double>(h);
}

int poisson_status(lbe_handle *h, lbe_stats *st, long long *kernels) {
  PoissonWork &w = h->pw;
  cudaError_t e = cudaMemcpyAsync(w.ctl_host, w.ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("poisson: ") + cudaGetErrorString(e);
    return LBE_ERR_CUDA;
  }
  const PoissonCtl &c = *w.ctl_host;
  if (st) {
    st->poisson_iters = c.total_iters;
    st->poisson_solves = (int)c.solves;
    st->poisson_max_iters = (int)(c.solve_iters > c.max_solve_iters ? c.solve_iters : c.max_solve_iters);
    st->poisson_residual = c.res;
  }
  // kernels of the graph path: reset + per round (residual, stencil,
  // correct) + per iteration (update, stencil)
  if (kernels && w.graph_ok) {
    // per solve: reset and the residual tests; per round that ran (every
    // test but the last of a solve): V-cycle, CG stencil, correction; per
    // iteration: update, V-cycle, stencil (a V-cycle only with multigrid)
    const long long vc = h->prm.precision == LBE_FP32 ? mg_kernels_per_cycle(h) : 0;
    *kernels = c.solves + c.total_rounds + (2 + vc) * (c.total_rounds - c.solves) + (2 + vc) * c.total_iters;
  }
  if (c.sticky_status == LBE_ERR_NOCONVERGE || c.status == LBE_ERR_NOCONVERGE) {
    h->err = "poisson: no convergence within poisson_max_iter";
    return LBE_ERR_NOCONVERGE;
  }
  if (c.sticky_status == LBE_ERR_NONFINITE || c.status == LBE_ERR_NONFINITE) {
    h->err = "poisson: non-finite residual";
    return LBE_ERR_NONFINITE;
  }
  return LBE_OK;
}

cudaError_t poisson_reset_stats(lbe_handle *h) { return cudaMemsetAsync(h->pw.ctl, 0, sizeof(PoissonCtl), h->stream); }


}  // namespace lbe
