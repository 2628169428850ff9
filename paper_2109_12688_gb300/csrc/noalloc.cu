// nadmm_spectral_solve_noalloc: the regulariser solve with its scratch in a
// fixed, library-owned device array instead of a caller workspace.
//
// Who needs it: code that may not allocate device memory itself.  Typical
// cases are a library embedded in a host application or framework that owns
// every device allocation through its own pool and forbids plug-ins from
// calling cudaMalloc, and latency-critical callers that cannot afford the
// implicit device synchronisation cudaMalloc/cudaFree may cause.  Such a
// caller still provides its input and output buffers; everything else comes
// from the static array below.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded reserves it until the process exits.  Host code cannot
// use the symbol as an address, so the first call on each device (with that
// device current) looks the address up with cudaGetSymbolAddress, raises the
// shared-memory limits of the pass kernels on that device, and caches the
// address; later calls reuse it.  The cached address belongs to the device's
// current context: after cudaDeviceReset (or a primary-context reset) the
// module is loaded again and the cached address must not be used, so such a
// reset and further calls of this entry point do not mix in one process.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/nadmm.h"
#include "nadmm_internal.h"
#include "plan.h"

namespace nadmm {
void set_last_error(const std::string& msg);  // defined in nadmm.cu
}

namespace {

using namespace nadmm;

constexpr size_t kStaticScratchBytes = size_t(24) << 20;  // 24 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

bool only_small_primes(int n) {
  for (int q : {2, 3, 5, 7})
    while (n % q == 0) n /= q;
  return n == 1;
}

int twiddle_count(const AxisPlan& p) {
  int n = 0;
  for (int i = 0; i < p.nst; ++i)
    if (p.m[i] > 1) n += (p.radix[i] - 1) * p.m[i];
  return n > 0 ? n : 1;
}

// Layout of the static array for one call.
struct StaticLayout {
  size_t spec, twx, twy, twz, posx, Kx, Ky, Kz, total;
};

StaticLayout layout_for(int nx, int ny, int nz, const AxisPlan& px, const AxisPlan& py,
                        const AxisPlan& pz) {
  StaticLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align256(o + bytes);
    return r;
  };
  L.spec = take((size_t)3 * (nx / 2 + 1) * ny * nz * sizeof(float2));
  L.twx = take((size_t)twiddle_count(px) * sizeof(float2));
  L.twy = take((size_t)twiddle_count(py) * sizeof(float2));
  L.twz = take((size_t)twiddle_count(pz) * sizeof(float2));
  L.posx = take((size_t)nx * sizeof(int));
  L.Kx = take((size_t)(nx / 2 + 1) * sizeof(float));
  L.Ky = take((size_t)ny * sizeof(float));
  L.Kz = take((size_t)nz * sizeof(float));
  L.total = o;
  return L;
}

// position that holds frequency k after the forward transform of plan p
__device__ int dev_freq_to_pos(const AxisPlan& p, int k) {
  int pos = 0;
  for (int i = 0; i < p.nst; ++i) {
    int d = k % p.radix[i];
    k /= p.radix[i];
    pos += d * p.m[i];
  }
  return pos;
}

// twiddle entry t of plan p: stage i holds w_{L_i}^{n1 k} at [(k-1) m_i + n1]
__device__ float2 dev_twiddle(const AxisPlan& p, int t) {
  for (int i = 0; i < p.nst; ++i) {
    if (p.m[i] <= 1) continue;
    int cnt = (p.radix[i] - 1) * p.m[i];
    if (t < cnt) {
      int k = t / p.m[i] + 1, n1 = t % p.m[i];
      long long e = (long long)n1 * k % p.L[i];
      double s, c;
      sincospi(-2.0 * (double)e / (double)p.L[i], &s, &c);
      return make_float2((float)c, (float)s);
    }
    t -= cnt;
  }
  return make_float2(1.0f, 0.0f);
}

__device__ float dev_sin2(int k, int n) {
  double s = sinpi((double)k / (double)n);
  return (float)(4.0 * s * s);
}

// Fill the FFT twiddles, the digit-reversal map and the per-axis symbols.
__global__ void k_fill_tables(AxisPlan px, AxisPlan py, AxisPlan pz, int ntx, int nty, int ntz,
                              float2* twx, float2* twy, float2* twz, int* posx, float* Kx,
                              float* Ky, float* Kz) {
  const int nx = px.n, ny = py.n, nz = pz.n, nkx = nx / 2 + 1;
  const int total = ntx + nty + ntz + nx + nkx + ny + nz;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int t = g;
    if (t < ntx) { twx[t] = dev_twiddle(px, t); continue; }
    t -= ntx;
    if (t < nty) { twy[t] = dev_twiddle(py, t); continue; }
    t -= nty;
    if (t < ntz) { twz[t] = dev_twiddle(pz, t); continue; }
    t -= ntz;
    if (t < nx) { posx[t] = dev_freq_to_pos(px, t); continue; }
    t -= nx;
    if (t < nkx) { Kx[t] = dev_sin2(t, nx); continue; }
    t -= nkx;
    if (t < ny) { Ky[dev_freq_to_pos(py, t)] = dev_sin2(t, ny); continue; }
    t -= ny;
    Kz[dev_freq_to_pos(pz, t)] = dev_sin2(t, nz);
  }
}

nadmm_status fail(nadmm_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

nadmm_status cuda_fail(cudaError_t e, const char* where) {
  return fail(NADMM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Set-up of the current device, once per device: the address of the static
// array, and the pass kernels' shared-memory limits raised to the maximum.
nadmm_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(NADMM_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch array");
    e = configure_admm_kernels_on_current_device();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return NADMM_OK;
}

}  // namespace

extern "C" nadmm_status nadmm_spectral_solve_noalloc(int32_t nx, int32_t ny, int32_t nz,
                                                     int32_t order_n, float lambda, float theta,
                                                     const float* y, float* w, void* stream) {
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 != 0 || ny % 2 != 0 || !only_small_primes(nx) ||
      !only_small_primes(ny) || !only_small_primes(nz))
    return fail(NADMM_ERR_UNSUPPORTED_SIZE,
                "dimensions must be >= 4, nx a multiple of 4, ny even, factors in {2,3,5,7}");
  if (order_n < 1 || order_n > 8 || !(lambda >= 0.0f) || !std::isfinite(lambda) ||
      !(theta > 0.0f) || !std::isfinite(theta))
    return fail(NADMM_ERR_INVALID_ARG, "need 1 <= order_n <= 8, finite lambda >= 0, theta > 0");
  if (!y || !w) return fail(NADMM_ERR_INVALID_ARG, "device pointer is NULL");
  if (((uintptr_t)y & 15u) || ((uintptr_t)w & 15u))
    return fail(NADMM_ERR_ALIGNMENT, "device pointer not 16-byte aligned");
  AxisPlan px, py, pz;
  if (!factor_axis(nx, px, true) || !factor_axis(ny, py, true, 16) || !factor_axis(nz, pz, true))
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "no radix plan for these dimensions");
  PlaneArgs a = {};
  a.px = px;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.theta = theta;
  a.eps = 1e-6f;
  a.data_term = 2;
  finish_plane_args(a);
  PencilArgs pa = {};
  pa.py = py;
  pa.pz = pz;
  pa.ny = ny;
  pa.nz = nz;
  pa.nkx = nx / 2 + 1;
  pa.order_n = order_n;
  pa.gamma = lambda / theta;
  pa.scale = (float)(1.0 / ((double)nx * ny * nz));
  finish_pencil_args(pa);
  if (plane_smem_max(a) > 227 * 1024 || pencil_smem_bytes(pa) > 227 * 1024)
    return fail(NADMM_ERR_UNSUPPORTED_SIZE,
                "a pass's shared-memory tile exceeds the 227 KB per CTA (nx too large)");
  if (nz > 256) return fail(NADMM_ERR_UNSUPPORTED_SIZE, "nz must be <= 256");
  const StaticLayout L = layout_for(nx, ny, nz, px, py, pz);
  if (L.total > kStaticScratchBytes)
    return fail(NADMM_ERR_UNSUPPORTED_SIZE,
                "grid needs " + std::to_string(L.total) +
                    " bytes of scratch; nadmm_spectral_solve_noalloc holds 25165824 (24 MiB)");

  void* base_v = nullptr;
  nadmm_status st = scratch_address(&base_v);
  if (st != NADMM_OK) return st;
  char* base = static_cast<char*>(base_v);
  cudaStream_t s = (cudaStream_t)stream;

  cudaError_t e = cudaSuccess;

  float2* twx = reinterpret_cast<float2*>(base + L.twx);
  float2* twy = reinterpret_cast<float2*>(base + L.twy);
  float2* twz = reinterpret_cast<float2*>(base + L.twz);
  int* posx = reinterpret_cast<int*>(base + L.posx);
  float* Kx = reinterpret_cast<float*>(base + L.Kx);
  float* Ky = reinterpret_cast<float*>(base + L.Ky);
  float* Kz = reinterpret_cast<float*>(base + L.Kz);
  const int ntx = twiddle_count(px), nty = twiddle_count(py), ntz = twiddle_count(pz);
  const int ntab = ntx + nty + ntz + nx + (nx / 2 + 1) + ny + nz;
  k_fill_tables<<<(ntab + 255) / 256, 256, 0, s>>>(px, py, pz, ntx, nty, ntz, twx, twy, twz, posx,
                                                   Kx, Ky, Kz);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "table fill");

  a.spec = reinterpret_cast<float2*>(base + L.spec);
  a.twx = twx;
  a.posx = posx;
  if (a.spec_tma) {
    e = encode_plane_map(a);
    if (e != cudaSuccess) return cuda_fail(e, "cuTensorMapEncodeTiled (plane)");
  }
  PlaneArgs fwd = a;
  fwd.y = nullptr;
  fwd.w_in = y;
  e = launch_plane(IN_FIELD, false, true, fwd, s);
  if (e == cudaSuccess) {
    pa.spec = a.spec;
    pa.twy = twy;
    pa.twz = twz;
    pa.Kx = Kx;
    pa.Ky = Ky;
    pa.Kz = Kz;
    e = encode_pencil_map(pa);
    if (e == cudaSuccess) e = launch_pencil(pa, s);
  }
  if (e == cudaSuccess) {
    PlaneArgs fin = a;
    fin.y = nullptr;
    fin.w_out = w;
    fin.b_out = nullptr;
    e = launch_plane(IN_SPEC, false, false, fin, s);
  }
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_spectral_solve_noalloc");
}
