// FP64 lattice kernels of one LBE time step (the "plain FP64" form).
//
//  * k_build_mask   per-node link mask of fluid neighbours (geometry set-up)
//  * k_init         uncharged capacitor, solvent at rest (Sec. "Potential and
//                   concentration profiles")
//  * k_sweep        fused ion link fluxes (Eq. LF1/LF2), solvent force from
//                   the link excess fluxes, D3Q19 BGK collision with Guo
//                   forcing (Eq. LBpop) and pull streaming with halfway
//                   bounce-back
//  * k_advect       cell-overlap advection of the solute by the velocity of
//                   the collision (scheme of Capuani et al., cited in the
//                   paper's Sec. "Lattice Boltzmann Electrokinetics")
//  * k_charge       induced electrode charge, Eq. Qelec
#include "lbe_internal.cuh"

namespace lbe {

namespace {

__device__ __forceinline__ long long nbr_i(const Geo &g, int x, int y, int z, int i) {
  return nbr(g, x, y, z, cx_of(i), cy_of(i), cz_of(i));
}

__global__ void k_build_mask(const Geo g, const uint8_t *__restrict__ id, uint32_t *__restrict__ mask) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  int x, y, z;
  coords(g, r, x, y, z);
  uint32_t m = id[r] == 0 ? kFluidBit : 0u;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    long long r2 = nbr_i(g, x, y, z, i);
    if (r2 >= 0 && id[r2] == 0) m |= 1u << (i - 1);
  }
  for (int sz = -1; sz <= 1; sz += 2)
    for (int sy = -1; sy <= 1; sy += 2)
      for (int sx = -1; sx <= 1; sx += 2) {
        long long r2 = nbr(g, x, y, z, sx, sy, sz);
        if (r2 >= 0 && id[r2] == 0) m |= 1u << corner_bit(sx, sy, sz);
      }
  mask[r] = m;
}

__global__ void k_init(const Geo g, int ns, const uint8_t *__restrict__ id,
                       const double *psi, double *__restrict__ f, double *__restrict__ n,
                       double *__restrict__ phi, double *__restrict__ u, double rb0, double rb1,
                       double rb2, double rb3) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const bool fl = id[r] == 0;
  const double rb[4] = {rb0, rb1, rb2, rb3};
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i * g.N + r] = fl ? w_of(i) : 0.0;
  for (int k = 0; k < ns; ++k) n[k * g.N + r] = fl ? rb[k] : 0.0;
  phi[r] = fl ? 0.0 : psi[id[r]];
  for (int a = 0; a < 3; ++a) u[a * g.N + r] = 0.0;
}

__global__ void k_init_phi(const Geo g, const uint8_t *__restrict__ id, const double *psi, double *__restrict__ phi) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  phi[r] = id[r] ? psi[id[r]] : 0.0;
}

__global__ void k_set_solid_phi(const Geo g, const uint8_t *__restrict__ id, const double *psi,
                                double *__restrict__ phi) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  if (id[r]) phi[r] = psi[id[r]];
}

// Link fluxes of Eq. LF2 in the relative form
//   j = -d/|c| * (1 + e^{-dmu})/2 * (n' e^{dmu} - n),
// dmu = z (phi' - phi - E.c); the solute update n* = n - sum_i j; the link
// excess flux g = j/d + (n' - n)/|c| summed into the solvent force
// F = (1/(2 A0)) sum_i c_i sum_k g.
__device__ __forceinline__ void ion_fluxes(const Geo &g, const Phys &P, long long r, int x, int y, int z,
                                           uint32_t m, const double *__restrict__ n,
                                           const double *__restrict__ phi, double *nstar_r, double F[3]) {
  const double phi0 = phi[r];
  double n0[LBE_MAX_SPECIES];
  for (int k = 0; k < P.ns; ++k) {
    n0[k] = n[k * g.N + r];
    nstar_r[k] = n0[k];
  }
  F[0] = F[1] = F[2] = 0.0;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    if (!(m & (1u << (i - 1)))) continue;
    const long long r2 = nbr_i(g, x, y, z, i);
    const double dphi = phi[r2] - phi0 - P.e_dot_c[i];
    double gsum = 0.0;
    for (int k = 0; k < P.ns; ++k) {
      const double n1 = n[k * g.N + r2];
      const double dmu = P.z[k] * dphi;
      const double e = exp(dmu);
      const double j = -P.d[k] * invlen_of(i) * 0.5 * (1.0 + 1.0 / e) * (n1 * e - n0[k]);
      nstar_r[k] -= j;
      gsum += j * P.inv_d[k] + (n1 - n0[k]) * invlen_of(i);
    }
    F[0] += cx_of(i) * gsum;
    F[1] += cy_of(i) * gsum;
    F[2] += cz_of(i) * gsum;
  }
  F[0] *= P.inv_2a0;
  F[1] *= P.inv_2a0;
  F[2] *= P.inv_2a0;
}

// Pull streaming: population i at r comes from r - c_i = r + c_opp(i) if that
// node is fluid, else it is the population opp(i) that left r towards the
// wall and was bounced back (halfway bounce-back).
__device__ __forceinline__ void gather(const Geo &g, long long r, int x, int y, int z, uint32_t m,
                                       const double *__restrict__ fin, double f[kQ]) {
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

template <bool FLOW>
__global__ void __launch_bounds__(kBlock) k_sweep(const Geo g, const Phys P, const uint32_t *__restrict__ mask,
                                                  const double *__restrict__ fin, double *__restrict__ fout,
                                                  const double *__restrict__ n, double *__restrict__ nstar,
                                                  const double *__restrict__ phi, double *__restrict__ u) {
  int x, y, z;
  long long r;
  if (!node_of(g, 1, 0, x, y, z, r)) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) return;
  double ns_r[LBE_MAX_SPECIES];
  double F[3];
  ion_fluxes(g, P, r, x, y, z, m, n, phi, ns_r, F);
  for (int k = 0; k < P.ns; ++k) nstar[k * g.N + r] = ns_r[k];
  if (!FLOW) return;

  double f[kQ];
  gather(g, r, x, y, z, m, fin, f);
  double rho = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    rho += f[i];
    mx += cx_of(i) * f[i];
    my += cy_of(i) * f[i];
    mz += cz_of(i) * f[i];
  }
  const double ux = (mx + 0.5 * F[0]) / rho, uy = (my + 0.5 * F[1]) / rho, uz = (mz + 0.5 * F[2]) / rho;
  u[r] = ux;
  u[g.N + r] = uy;
  u[2 * g.N + r] = uz;
  const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const double cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    const double feq = w_of(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    const double cF = cx_of(i) * F[0] + cy_of(i) * F[1] + cz_of(i) * F[2];
    const double uF = ux * F[0] + uy * F[1] + uz * F[2];
    const double src = P.guo * w_of(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
    fout[i * g.N + r] = f[i] - P.omega * (f[i] - feq) + src;
  }
}

// Cell-overlap advection (pull form): node r collects, from every source
// q = r - s (s in {-1,0,1}^3) that is fluid, the share of q's solute whose
// displaced cell overlaps r; plus the shares of its own solute that would
// have landed on solid nodes.
__device__ __forceinline__ double ov(int s, double u) {
  return s == 0 ? 1.0 - fabs(u) : (s > 0 ? fmax(u, 0.0) : fmax(-u, 0.0));
}

__device__ __forceinline__ int dir_bit(int dx, int dy, int dz) {
  // bit of the mask for the neighbour at offset (dx,dy,dz) != 0
  if (dx != 0 && dy != 0 && dz != 0) return corner_bit(dx, dy, dz);
#pragma unroll
  for (int i = 1; i < kQ; ++i)
    if (cx_of(i) == dx && cy_of(i) == dy && cz_of(i) == dz) return i - 1;
  return -1;
}

__global__ void __launch_bounds__(kBlock) k_advect(const Geo g, int ns, const uint32_t *__restrict__ mask,
                                                   const double *__restrict__ nin, const double *__restrict__ u,
                                                   double *__restrict__ nout) {
  int x, y, z;
  long long r;
  if (!node_of(g, 1, 0, x, y, z, r)) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int k = 0; k < ns; ++k) nout[k * g.N + r] = 0.0;
    return;
  }
  double acc[LBE_MAX_SPECIES] = {0.0, 0.0, 0.0, 0.0};
  const double ux = u[r], uy = u[g.N + r], uz = u[2 * g.N + r];
  double keep = 0.0;  // own shares bound for solid neighbours
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) {
          const double w = ov(0, ux) * ov(0, uy) * ov(0, uz);
          for (int k = 0; k < ns; ++k) acc[k] += w * nin[k * g.N + r];
          continue;
        }
        // source q = r - s exists as fluid iff the neighbour at -s is fluid
        if (m & (1u << dir_bit(-dx, -dy, -dz))) {
          const long long q = nbr(g, x, y, z, -dx, -dy, -dz);
          const double w = ov(dx, u[q]) * ov(dy, u[g.N + q]) * ov(dz, u[2 * g.N + q]);
          if (w != 0.0)
            for (int k = 0; k < ns; ++k) acc[k] += w * nin[k * g.N + q];
        }
        if (!(m & (1u << dir_bit(dx, dy, dz)))) keep += ov(dx, ux) * ov(dy, uy) * ov(dz, uz);
      }
  for (int k = 0; k < ns; ++k) nout[k * g.N + r] = acc[k] + keep * nin[k * g.N + r];
}

// Velocity and density of the current state, (sum f c + F/2)/rho with F from
// the current n and phi.
__global__ void k_moments(const Geo g, const Phys P, int flow, const uint32_t *__restrict__ mask,
                          const double *__restrict__ fin, const double *__restrict__ n,
                          const double *__restrict__ phi, double *__restrict__ rho_out,
                          double *__restrict__ u_out) {
  int x, y, z;
  long long r;
  if (!node_of(g, 1, 0, x, y, z, r)) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    if (rho_out) rho_out[r] = 0.0;
    if (u_out) u_out[r] = u_out[g.N + r] = u_out[2 * g.N + r] = 0.0;
    return;
  }
  double ns_r[LBE_MAX_SPECIES], F[3];
  ion_fluxes(g, P, r, x, y, z, m, n, phi, ns_r, F);
  double f[kQ];
  gather(g, r, x, y, z, m, fin, f);
  double rho = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
  for (int i = 0; i < kQ; ++i) {
    rho += f[i];
    mx += cx_of(i) * f[i];
    my += cy_of(i) * f[i];
    mz += cz_of(i) * f[i];
  }
  if (rho_out) rho_out[r] = rho;
  if (u_out) {
    u_out[r] = flow ? (mx + 0.5 * F[0]) / rho : 0.0;
    u_out[g.N + r] = flow ? (my + 0.5 * F[1]) / rho : 0.0;
    u_out[2 * g.N + r] = flow ? (mz + 0.5 * F[2]) / rho : 0.0;
  }
}

__global__ void k_gather_f(const Geo g, const uint32_t *__restrict__ mask, const double *__restrict__ fin,
                           double *__restrict__ out) {
  int x, y, z;
  long long r;
  if (!node_of(g, 1, 0, x, y, z, r)) return;
  const uint32_t m = mask[r];
  if (!(m & kFluidBit)) {
    for (int i = 0; i < kQ; ++i) out[i * g.N + r] = 0.0;
    return;
  }
  double f[kQ];
  gather(g, r, x, y, z, m, fin, f);
  for (int i = 0; i < kQ; ++i) out[i * g.N + r] = f[i];
}

// Eq. Qelec, per block and electrode: -eps * sum over the block's electrode
// nodes of the modified Laplacian over links to fluid (factor 2 on every
// such boundary link).  Partials are summed in block order by k_charge_final.
__global__ void __launch_bounds__(kBlock) k_charge_partial(const Geo g, const Phys P, int n_elec,
                                                           const uint8_t *__restrict__ id,
                                                           const uint32_t *__restrict__ mask,
                                                           const double *__restrict__ phi,
                                                           double *__restrict__ part) {
  __shared__ double sh[kBlock / 32][LBE_MAX_ELECTRODES];
  double acc[LBE_MAX_ELECTRODES];
  for (int e = 0; e < n_elec; ++e) acc[e] = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const int e = id[r];
    if (!e) continue;
    const uint32_t m = mask[r];
    if (!(m & ((1u << 18) - 1))) continue;
    int x, y, z;
    coords(g, r, x, y, z);
    const double p0 = phi[r];
    double s = 0.0;
    for (int i = 1; i < kQ; ++i)
      if (m & (1u << (i - 1))) s += lapc_of(i) * P.solid_factor * (phi[nbr_i(g, x, y, z, i)] - p0);
    for (int k = 0; k < n_elec; ++k)
      if (k == e - 1) acc[k] += -P.eps * s;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = 0; e < n_elec; ++e) {
    double v = acc[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][e] = v;
  }
  __syncthreads();
  if (threadIdx.x < n_elec) {
    double v = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) v += sh[w][threadIdx.x];
    part[(long long)blockIdx.x * n_elec + threadIdx.x] = v;
  }
}

__global__ void k_charge_final(int nblk, int n_elec, const double *__restrict__ part, double *__restrict__ q) {
  // one warp per electrode; lanes stride the partials, then a fixed tree
  const int e = blockIdx.x;
  if (e >= n_elec) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) v += part[(long long)b * n_elec + e];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) q[e] = v;
}

// per-node term of Eq. Qelec (the map behind lbe_induced_charge)
__global__ void k_charge_node(const Geo g, const Phys P, const uint8_t *__restrict__ id,
                              const uint32_t *__restrict__ mask, const double *__restrict__ phi,
                              double *__restrict__ out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.N) return;
  const uint32_t m = mask[r];
  if (!id[r] || !(m & ((1u << 18) - 1))) {
    out[r] = 0.0;
    return;
  }
  int x, y, z;
  coords(g, r, x, y, z);
  double s = 0.0;
  for (int i = 1; i < kQ; ++i)
    if (m & (1u << (i - 1))) s += lapc_of(i) * P.solid_factor * (phi[nbr_i(g, x, y, z, i)] - phi[r]);
  out[r] = -P.eps * s;
}

inline unsigned grid_for(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }
#define LAUNCH3(h) make_launch((h)->geo).grid, make_launch((h)->geo).block

}  // namespace

cudaError_t launch_build_mask(const Geo &g, const uint8_t *id, uint32_t *mask, cudaStream_t s) {
  k_build_mask<<<grid_for(g.N), kBlock, 0, s>>>(g, id, mask);
  return cudaGetLastError();
}

// Electrode potentials are staged from a host stack array: an H2D copy from
// pageable memory returns only once the source has been consumed.
static cudaError_t stage_psi(lbe_handle *h) {
  double tmp[LBE_MAX_ELECTRODES + 1];
  tmp[0] = 0.0;
  for (int e = 0; e < h->n_elec; ++e) tmp[e + 1] = h->psi[e];
  return cudaMemcpyAsync(h->psi_dev, tmp, sizeof(double) * (h->n_elec + 1), cudaMemcpyHostToDevice,
                         h->stream);
}

cudaError_t launch_init_state(lbe_handle *h) {
  const double *rb = h->prm.rho_bulk;
  cudaError_t err = stage_psi(h);
  if (err != cudaSuccess) return err;
  k_init<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->prm.nspecies, h->id, h->psi_dev,
                                                        h->f[h->cur], h->n, h->phi, h->u, rb[0], rb[1],
                                                        rb[2], rb[3]);
  return cudaGetLastError();
}

cudaError_t launch_init_phi(lbe_handle *h) {
  cudaError_t err = stage_psi(h);
  if (err != cudaSuccess) return err;
  k_init_phi<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->id, h->psi_dev, h->phi);
  return cudaGetLastError();
}

cudaError_t launch_set_solid_phi(lbe_handle *h) {
  cudaError_t err = stage_psi(h);
  if (err != cudaSuccess) return err;
  k_set_solid_phi<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->id, h->psi_dev, h->phi);
  return cudaGetLastError();
}

cudaError_t launch_sweep(lbe_handle *h) {
  const int nxt = h->cur ^ 1;
  if (h->prm.flow)
    k_sweep<true><<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->phys, h->mask, h->f[h->cur],
                                                                 h->f[nxt], h->n, h->nstar, h->phi, h->u);
  else
    k_sweep<false><<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->phys, h->mask, h->f[h->cur],
                                                                  h->f[nxt], h->n, h->nstar, h->phi, h->u);
  if (h->prm.flow) h->cur = nxt;
  return cudaGetLastError();
}

cudaError_t launch_advect(lbe_handle *h) {
  k_advect<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->prm.nspecies, h->mask, h->nstar, h->u, h->n);
  return cudaGetLastError();
}

cudaError_t launch_moments(lbe_handle *h, double *rho_out, double *u_out) {
  k_moments<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->phys, h->prm.flow, h->mask,
                                                           h->f[h->cur], h->n, h->phi, rho_out, u_out);
  return cudaGetLastError();
}

cudaError_t launch_gather_f(lbe_handle *h, double *out) {
  k_gather_f<<<LAUNCH3(h), 0, h->stream>>>(h->geo, h->mask, h->f[h->cur], out);
  return cudaGetLastError();
}

cudaError_t launch_charge_node(lbe_handle *h, double *out) {
  k_charge_node<<<grid_for(h->geo.N), kBlock, 0, h->stream>>>(h->geo, h->phys, h->id, h->mask, h->phi, out);
  return cudaGetLastError();
}

cudaError_t launch_charge(lbe_handle *h) {
  k_charge_partial<<<h->qblk, kBlock, 0, h->stream>>>(h->geo, h->phys, h->n_elec, h->id, h->mask, h->phi,
                                                       h->qpart);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_charge_final<<<h->n_elec, 32, 0, h->stream>>>(h->qblk, h->n_elec, h->qpart, h->qout);
  return cudaGetLastError();
}

}  // namespace lbe
