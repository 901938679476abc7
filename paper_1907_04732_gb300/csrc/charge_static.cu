// Induced electrode charge from caller-owned buffers, with no device memory
// allocated by the call (declaration and contract in include/lbe.h).
//
// The per-block partial sums live in a file-scope device array instead of a
// cudaMalloc'd buffer.  Host code cannot pass that array's name to a kernel
// (on the host it is only a stand-in symbol), so its device address is looked
// up once per device with cudaGetSymbolAddress and cached.
#include <mutex>
#include <string>

#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int kStaticBlocks = 1024;  // grid-stride blocks; partials per electrode
constexpr int kMaxDevices = 64;

// 1024 x 16 doubles = 128 KiB on every device that loads this library
static __device__ __align__(256) double g_charge_scratch[kStaticBlocks * LBE_MAX_ELECTRODES];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

__global__ void __launch_bounds__(kBlock) k_charge_static_partial(const Geo g, double eps, int n_elec,
                                                                  const uint8_t *__restrict__ id,
                                                                  const double *__restrict__ phi,
                                                                  double *__restrict__ part) {
  __shared__ double sh[kBlock / 32][LBE_MAX_ELECTRODES];
  double acc[LBE_MAX_ELECTRODES];
  for (int e = 0; e < LBE_MAX_ELECTRODES; ++e) acc[e] = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
       r += (long long)gridDim.x * blockDim.x) {
    const int e = id[r];
    if (!e) continue;
    int x, y, z;
    coords(g, r, x, y, z);
    const double p0 = phi[r];
    double s = 0.0;
    // Eq. Qelec: modified Laplacian over the links to fluid nodes, each
    // boundary link doubled
    for (int i = 1; i < kQ; ++i) {
      const long long r2 = nbr(g, x, y, z, cx_of(i), cy_of(i), cz_of(i));
      if (r2 < 0 || id[r2] != 0) continue;
      s += lapc_of(i) * 2.0 * (phi[r2] - p0);
    }
    for (int k = 0; k < LBE_MAX_ELECTRODES; ++k)
      if (k == e - 1) acc[k] += -eps * s;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = 0; e < n_elec; ++e) {
    double v = acc[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][e] = v;
  }
  __syncthreads();
  // every call rewrites all partials it later reads: nothing to clear
  if (threadIdx.x < n_elec) {
    double v = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) v += sh[w][threadIdx.x];
    part[(long long)blockIdx.x * n_elec + threadIdx.x] = v;
  }
}

__global__ void k_charge_static_final(int nblk, int n_elec, const double *__restrict__ part, double *__restrict__ q) {
  const int e = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) v += part[(long long)b * n_elec + e];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) q[e] = v;
}

int fail_static(int code, const char *msg) {
  set_static_error(msg);
  return code;
}

}  // namespace

}  // namespace lbe

extern "C" int lbe_induced_charge_static(const double *phi, const uint8_t *node_id, int nx, int ny, int nz,
                                         const int *periodic, double bjerrum, int n_electrodes, double *q_out,
                                         void *cuda_stream) {
  using namespace lbe;
  if (!phi || !node_id || !periodic || !q_out) return fail_static(LBE_ERR_ARG, "induced_charge_static: NULL pointer");
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31))
    return fail_static(LBE_ERR_ARG, "induced_charge_static: lattice size out of range");
  if (n_electrodes < 1 || n_electrodes > LBE_MAX_ELECTRODES)
    return fail_static(LBE_ERR_ARG,
                       "induced_charge_static: n_electrodes exceeds the static scratch (max LBE_MAX_ELECTRODES)");
  if (!(bjerrum > 0.0)) return fail_static(LBE_ERR_ARG, "induced_charge_static: bjerrum must be > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_static(LBE_ERR_CUDA, "induced_charge_static: no current CUDA device");
  double *part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      // first call on this device: the device address of the static array
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_charge_scratch);
      if (e != cudaSuccess) return fail_static(LBE_ERR_CUDA, "induced_charge_static: cudaGetSymbolAddress failed");
      g_scratch_addr[dev] = (double *)p;
    }
    part = g_scratch_addr[dev];
  }
  const Geo g{nx, ny, nz, periodic[0] != 0, periodic[1] != 0, periodic[2] != 0, (long long)nx * ny * nz};
  const long long want = (g.N + kBlock - 1) / kBlock;
  const int nblk = (int)(want < kStaticBlocks ? want : kStaticBlocks);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_charge_static_partial<<<nblk, kBlock, 0, st>>>(g, 1.0 / (4.0 * M_PI * bjerrum), n_electrodes, node_id, phi, part);
  k_charge_static_final<<<n_electrodes, 32, 0, st>>>(nblk, n_electrodes, part, q_out);
  if (cudaGetLastError() != cudaSuccess) return fail_static(LBE_ERR_CUDA, "induced_charge_static: launch failed");
  return LBE_OK;
}
