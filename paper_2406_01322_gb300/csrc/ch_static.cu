// Allocation-free forward transform: ch_transform_forward_noalloc.
//
// Some callers cannot allocate device memory at the moment they need a transform: plug-ins
// hosted by an application whose memory pool already owns the device's memory, or
// fixed-latency loops that must not enter the allocator.  This entry point serves them: it
// computes the same physical -> spectral transform as ch_transform_forward (Fourier in x and y,
// then the Chebyshev DCT-I, with the handle's radix schedules) without a handle and without
// allocating.  Its working memory is one file-scope device array of kStaticScratchBytes
// (64 MiB), which every GPU that loads this library holds until the process exits.  Twiddles are
// computed on the device (sincospi) rather than rounded from extended-precision host values, so
// the result equals the handle's to rounding, not bit for bit.
//
// Set-up: the first call on a device (with that device current) looks up the array's device
// address with cudaGetSymbolAddress; later calls reuse it.  The first call for a grid larger
// than any before may raise a kernel's dynamic shared-memory limit.  Make both before any stream
// capture.  Every call shares the array and leaves its contents behind; nothing in it needs to
// start at zero (each stage writes every element the next stage reads).  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array.
#include <mutex>

#include "../../include/ch_flow.h"
#include "ch_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// twiddles exp(-2 pi i t / n), t < n
__global__ void static_twiddles_kernel(double2* tw, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_double2(c, -s);
  }
}

// (cos(pi j / n), sin(pi j / n)), j < n: the Chebyshev transform's pre/post factors
__global__ void static_cs_kernel(double2* cs, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    double s, c;
    sincospi((double)t / (double)n, &s, &c);
    cs[t] = make_double2(c, s);
  }
}

// device address of the scratch array for the current device, set up once per device
int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return CH_OK;
}

}  // namespace

extern "C" size_t ch_noalloc_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int ch_transform_forward_noalloc(int nx, int ny, int nz, const double* phys,
                                            double* spec, void* stream) {
  if (!phys || !spec) return CH_ERR_ARG;
  if (chf::check_sizes(nx, ny, nz) != CH_OK) return CH_ERR_SIZE;
  chf::GridDev g = {};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.N = nz - 1;
  g.Mx = nx / 2;
  g.Px = 3 * nx / 2;
  g.Py = 3 * ny / 2;
  // the forward transform does not depend on the box size; the library's default box
  g.lx = 4.0 * 3.14159265358979323846;
  g.ly = 2.0 * 3.14159265358979323846;
  const long long fs = (long long)g.Mx * ny * nz;
  // scratch layout: x, y, z twiddles, then two (Mx, Ny, Nz) complex fields
  const size_t b_tx = round256((size_t)nx * sizeof(double2));
  const size_t b_ty = round256((size_t)ny * sizeof(double2));
  const size_t b_tz = round256((size_t)2 * g.N * sizeof(double2));  // N twiddles + N cos/sin
  const size_t b_f = round256((size_t)fs * sizeof(double2));
  if (b_tx + b_ty + b_tz + 2 * b_f > kStaticScratchBytes) return CH_ERR_SIZE;
  unsigned char* base = nullptr;
  int st = scratch_for_current_device(&base);
  if (st != CH_OK) return st;
  double2* tx = reinterpret_cast<double2*>(base);
  double2* ty = reinterpret_cast<double2*>(base + b_tx);
  double2* tz = reinterpret_cast<double2*>(base + b_tx + b_ty);
  double2* A = reinterpret_cast<double2*>(base + b_tx + b_ty + b_tz);
  double2* B = reinterpret_cast<double2*>(base + b_tx + b_ty + b_tz + b_f);
  chf::FftPlan px, py, pz;
  // the schedules of the handle's transform: default ones for the unpadded x and y lengths,
  // maximal radix-8 for the Chebyshev lines
  if (!chf::make_radices(nx, &px) || !chf::make_radices(ny, &py) ||
      !chf::make_radices_style(g.N, 2, &pz))
    return CH_ERR_SIZE;
  px.tw = tx;
  py.tw = ty;
  pz.tw = tz;
  g.zcs = tz + g.N;
  cudaStream_t s = (cudaStream_t)stream;
  static_twiddles_kernel<<<(nx + 255) / 256, 256, 0, s>>>(tx, nx);
  static_twiddles_kernel<<<(ny + 255) / 256, 256, 0, s>>>(ty, ny);
  static_twiddles_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(tz, g.N);
  static_cs_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(tz + g.N, g.N);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = chf::launch_x_r2c(g, phys, A, 1, (long long)nx * ny * nz, fs, px, s);
  if (e == cudaSuccess)
    e = chf::launch_ypass(0, 0, g, ny, A, B, 1, fs, fs, 1.0 / ((double)nx * (double)ny), py, s);
  if (e == cudaSuccess) e = chf::launch_dct_lines(0, 0, g, B, (double2*)spec, 1, fs, pz, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  return CH_OK;
}
