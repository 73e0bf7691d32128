// sph_noalloc.cu -- cell sort of a caller's point set that allocates no
// device memory (declared in include/sph.h as sph_cell_sort_noalloc).
//
// It computes what the cell sort inside sph_step computes (cell keys of
// cell size 2h, stable LSD radix sort, cell offsets) with the multi-launch
// radix sort of sph_sort.cu, whose launches never wait on one another, and
// its scratch lives in one file-scope static device array instead of memory
// the context allocates.  Callers that must not allocate -- code running while a CUDA
// stream is being captured into a graph, or a host application whose device
// memory is reserved up front and may not grow during a run -- can call it
// with their own input and output buffers only.
//
// Limits and sharing:
//  * at most SPH_NOALLOC_MAX_POINTS points per call (larger n is rejected
//    with SPH_ERR_ARG);
//  * the array (about 9.4 MB) exists on every GPU that loads the library,
//    for the life of the process;
//  * every call on a device uses the same array and leaves its contents
//    behind; everything a call reads is written earlier in the same call,
//    so no clearing is needed, but calls that overlap on the GPU (different
//    streams without ordering) race on it;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (host code must not use the array's name as a
//    device pointer); make that first call before any stream capture.  The
//    address is kept for the life of the process: after cudaDeviceReset the
//    module holding the array is loaded anew and the kept address is stale,
//    so the call is not valid across a device reset;
//  * errors set the message of sph_last_error(); a CUDA error already
//    pending on the thread when the call starts is reported as such (the
//    call then launches nothing) instead of being taken for its own.
#include <cmath>
#include <mutex>
#include <string>

#include "sph_internal.cuh"

namespace {

constexpr int kMaxPoints = SPH_NOALLOC_MAX_POINTS;
constexpr int kTile = 2048;  // radix tile of sph_sort.cu
constexpr int kMaxBlocks = (kMaxPoints + kTile - 1) / kTile;

// digit histograms of up to 10-bit digits plus their scan chunk totals
constexpr int kHistWords = (1 << 10) * kMaxBlocks + ((1 << 10) * kMaxBlocks + 2047) / 2048 + 1;

// keys[2][max], vals[2][max], histogram, counters
struct Scratch {
  uint32_t keys[2][kMaxPoints];
  uint32_t vals[2][kMaxPoints];
  uint32_t hist[kHistWords];
  int32_t count;
  int32_t nlive;
};

static __device__ __align__(256) Scratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
Scratch *g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the array on the current device, looked up once per
// device (the symbol's name in host code is not a device address)
int scratch_for_current_device(Scratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sphk::set_error(SPH_ERR_CUDA, "sph_cell_sort_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return sphk::set_error(SPH_ERR_CUDA, (std::string("sph_cell_sort_noalloc: cudaGetSymbolAddress: ") +
                                            cudaGetErrorString(e)).c_str());
    g_scratch_ptr[dev] = (Scratch *)p;
  }
  *out = g_scratch_ptr[dev];
  return SPH_OK;
}

struct Grid {
  int dim;
  int nc[3];
  double lo[3], cs;
};

__global__ void k_noalloc_keys(const double *__restrict__ pos, int n, Grid g, Scratch *s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) s->count = n;
  if (i >= n) return;
  uint32_t c[3] = {0, 0, 0};
  for (int a = 0; a < g.dim; ++a) {
    double f = floor(sphk::ddiv(sphk::dsub(pos[3 * i + a], g.lo[a]), g.cs));
    if (!(f >= 0.0))
      c[a] = 0;
    else if (f >= (double)g.nc[a])
      c[a] = (uint32_t)g.nc[a] - 1;
    else
      c[a] = (uint32_t)f;
  }
  s->keys[0][i] = (c[2] * (uint32_t)g.nc[1] + c[1]) * (uint32_t)g.nc[0] + c[0];
  s->vals[0][i] = (uint32_t)i;
}

__global__ void k_noalloc_copy(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

}  // namespace

extern "C" int sph_cell_sort_noalloc(const sph_config *cfg, const double *pos, int32_t n, uint32_t *order,
                                     uint32_t *cell_start, int64_t cell_start_len, int64_t *ncell_out,
                                     void *stream) {
  auto arg = [](const char *why) { return sphk::set_error(SPH_ERR_ARG, why); };
  if (!cfg || n < 0 || (n > 0 && (!pos || !order)) || !cell_start)
    return arg("sph_cell_sort_noalloc: NULL pointer or negative n");
  if (n > kMaxPoints) return arg("sph_cell_sort_noalloc: n above SPH_NOALLOC_MAX_POINTS");
  if ((cfg->dim != 2 && cfg->dim != 3) || !(cfg->h > 0)) return arg("sph_cell_sort_noalloc: bad dim or h");
  Grid g{};
  g.dim = cfg->dim;
  g.cs = 2.0 * cfg->h;
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = 1;
    g.lo[a] = cfg->domain_lo[a];
    if (a < cfg->dim) {
      double L = cfg->domain_hi[a] - cfg->domain_lo[a];
      if (!(L > 0)) return arg("sph_cell_sort_noalloc: domain_hi must exceed domain_lo");
      double f = std::floor(L / g.cs);
      if (f > 1.0e6) return arg("sph_cell_sort_noalloc: cell grid too large");
      g.nc[a] = (f >= 1.0) ? (int)f : 1;
    }
    ncell *= g.nc[a];
  }
  if (ncell_out) *ncell_out = ncell;
  if (ncell >= (1ll << 31)) return arg("sph_cell_sort_noalloc: cell grid too large");
  if (cell_start_len < ncell + 1) return arg("sph_cell_sort_noalloc: cell_start shorter than ncell + 1");
  {
    const cudaError_t pre = cudaPeekAtLastError();
    if (pre != cudaSuccess)
      return sphk::set_error(SPH_ERR_CUDA, (std::string("sph_cell_sort_noalloc: CUDA error pending before the call: ") +
                                            cudaGetErrorString(pre)).c_str());
  }
  Scratch *s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (n + 255) / 256 > 0 ? (n + 255) / 256 : 1;
  k_noalloc_keys<<<blocks, 256, 0, st>>>(pos, n, g, s);
  int bits = 1;
  while ((1ll << bits) <= ncell) ++bits;
  sphk::SortTemp tmp{s->hist, kMaxBlocks};
  uint32_t *kr = nullptr, *vr = nullptr;
  sphk::radix_sort(s->keys[0], s->vals[0], s->keys[1], s->vals[1], &s->count, n > 0 ? n : 1, bits, tmp, st, &kr,
                   &vr);
  sphk::cell_offsets(kr, &s->count, (uint32_t)ncell, cell_start, &s->nlive, st);
  if (n > 0) k_noalloc_copy<<<blocks, 256, 0, st>>>(vr, order, n);
  // nothing was pending at entry, so an error here is one of this call's launches
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return sphk::set_error(SPH_ERR_CUDA, (std::string("sph_cell_sort_noalloc: ") + cudaGetErrorString(e)).c_str());
  return SPH_OK;
}
