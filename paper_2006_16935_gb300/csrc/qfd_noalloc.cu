// qfd_energy_noalloc: the Rayleigh energy of a caller's device lattice
// computed without allocating any device memory.
//
// Some callers cannot allocate: a serving process that hands its whole
// device-memory budget to its own pool up front, or code on a latency-critical
// path where a cudaMalloc could fail or stall the device, still wants to
// evaluate <psi|H_K + V|psi>.  For them the work lattice, the per-CTA partial
// sums, the twiddle and kinetic tables and the result scalars live in one
// file-scope static device array of fixed size, which every GPU that loads
// this library holds until the process exits.  Its size bounds the lattice:
// N^3 complex128 sites of work space, so N <= 128.
//
// The array is shared by all calls and keeps the last call's contents.
// Nothing in it has to start at zero: every pass overwrites what it reads
// later (each CTA writes its own partial, the reductions write the scalars).
// Calls that overlap on the GPU (on different streams, or from different host
// threads) race on the array: serialise them.
//
// Set-up: the device address of the array is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// it; make that first call before any stream capture.  The address lives as
// long as the device's context: after a cudaDeviceReset the entry point must
// not be called again on that device in the same process.
//
// Only the FFT kinetic terms (kinetic 1..3) are accepted: the energy's
// kinetic part is the Parseval sum of Eqs. (HK1)-(HK3).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "qfd.h"
#include "qfd_kernels.cuh"
#include "qfd_launch.h"

namespace {

using namespace qfd;

constexpr int64_t NOALLOC_MAX_N = 128;
constexpr size_t ALIGN = 256;
constexpr size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }
// layout of the static array (byte offsets)
constexpr size_t OFF_W = 0;
constexpr size_t SZ_W = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N * sizeof(double2);
constexpr size_t MAX_PART = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N;  // >= CTAs of any reducing pass
constexpr size_t OFF_PA = align_up(OFF_W + SZ_W);                   // 2 partials per CTA (norm, <V>)
constexpr size_t OFF_PC = align_up(OFF_PA + 2 * MAX_PART * sizeof(double));
constexpr size_t OFF_TW = align_up(OFF_PC + MAX_PART * sizeof(double));
constexpr size_t OFF_KT = align_up(OFF_TW + 3 * NOALLOC_MAX_N * sizeof(double2));  // + the scaled block
constexpr size_t OFF_SC = align_up(OFF_KT + NOALLOC_MAX_N * sizeof(double));
constexpr size_t SCRATCH_BYTES = align_up(OFF_SC + 4 * sizeof(double));

__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// Sums the per-CTA partials in a fixed order: out[0] = E, out[1] = sum |psi|^2.
__global__ void __launch_bounds__(1024)
k_noalloc_energy(const double* __restrict__ pa, int na, const double* __restrict__ pc, int nc, double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ double sums[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 3; ++q) {
    const double* p = q == 2 ? pc : pa + (size_t)q * na;
    const int cnt = q == 2 ? nc : na;
    double x = 0.0;
    for (int i = threadIdx.x; i < cnt; i += 1024) x += p[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
      double y = red[lane];
      for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
      if (lane == 0) sums[q] = y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = (sums[2] + sums[1]) / sums[0];
    out[1] = sums[0];
  }
}

// exp(-2 pi i e / n) with the angle reduced to the first octant in integers.
void twiddle(int64_t e, int64_t n, double* c, double* s) {
  const int64_t q = (4 * e) / n, rem = 4 * e - q * n;
  double cp, sp;
  if (2 * rem <= n) {
    const double phi = (M_PI / 2) * (double)rem / (double)n;
    cp = std::cos(phi);
    sp = std::sin(phi);
  } else {
    const double phi = (M_PI / 2) * (double)(n - rem) / (double)n;
    cp = std::sin(phi);
    sp = std::cos(phi);
  }
  const double ct[4] = {cp, -sp, -cp, sp}, st[4] = {sp, cp, -sp, -cp};
  *c = ct[q];
  *s = -st[q];
}

unsigned char* scratch_for_current_device(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= MAX_DEVICES) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" qfd_status qfd_energy_noalloc(const double* psi, const double* V, int64_t n, double a, double mass,
                                         int kinetic, int rest_mass, void* stream, double* E, double* norm2) {
  if (!psi || !V || !(a > 0) || !(mass > 0) || kinetic < 1 || kinetic > 3 || (rest_mass != 0 && rest_mass != 1))
    return QFD_ERR_ARG;
  if (!supported_n(n) || n > NOALLOC_MAX_N) return QFD_ERR_ARG;  // the static scratch holds N <= 128
  cudaError_t err = cudaSuccess;
  unsigned char* base = scratch_for_current_device(&err);
  if (!base) return QFD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  // per-axis tables of Eqs. (HK1)-(HK3) and the twiddles, copied into the array
  double2 tw[3 * NOALLOC_MAX_N];
  double kt[NOALLOC_MAX_N];
  for (int64_t j = 0; j < n; ++j) {
    double c, s;
    twiddle(j, n, &c, &s);
    tw[j] = double2{c, s};
    const int64_t m = j <= n / 2 ? j : j - n;
    if (kinetic == 1) {
      const double k = 2.0 * M_PI * (double)m / (double)n;
      kt[j] = k * k;
    } else {
      const double sn = std::sin(M_PI * (double)(m < 0 ? -m : m) / (double)n);
      kt[j] = 4.0 * sn * sn;
    }
  }
  const double n3d = (double)n * (double)n * (double)n;
  KinParams kin{};
  kin.kinterm = kinetic;
  kin.pref = 1.0 / (2.0 * a * a * mass * n3d);
  kin.am2 = (a * mass) * (a * mass);
  kin.inv_a_n3 = 1.0 / (a * n3d);
  kin.m0_n3 = rest_mass ? 0.0 : mass / n3d;
  scaled_twiddle_table(n, tw, tw + n);
  if ((err = cudaMemcpyAsync(base + OFF_TW, tw, 3 * n * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (err = cudaMemcpyAsync(base + OFF_KT, kt, n * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return QFD_ERR_CUDA;

  if ((size_t)max_partials<F64>(n) > MAX_PART) return QFD_ERR_ARG;
  LaunchArgs la;
  la.n = n;
  la.W = base + OFF_W;
  la.src = psi;
  la.V = V;
  la.tw = base + OFF_TW;
  la.ktab = base + OFF_KT;
  la.kin = &kin;
  la.stream = st;
  int na = 0, nc = 0;
  la.part = reinterpret_cast<double*>(base + OFF_PA);
  la.stats = STATS_FULL;
  if (launch_forward_x<F64>(la, &na) != cudaSuccess) return QFD_ERR_CUDA;
  if (launch_fft_y<F64>(la, -1) != cudaSuccess) return QFD_ERR_CUDA;
  la.part = reinterpret_cast<double*>(base + OFF_PC);
  la.stats = 1;  // Parseval sum of T |psi~|^2
  if (launch_zpass<F64>(la, &nc) != cudaSuccess) return QFD_ERR_CUDA;
  double* sc = reinterpret_cast<double*>(base + OFF_SC);
  k_noalloc_energy<<<1, 1024, 0, st>>>(reinterpret_cast<const double*>(base + OFF_PA), na,
                                       reinterpret_cast<const double*>(base + OFF_PC), nc, sc);
  if (cudaGetLastError() != cudaSuccess) return QFD_ERR_CUDA;
  double out[2];
  if (cudaMemcpyAsync(out, sc, sizeof(out), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return QFD_ERR_CUDA;
  if (E) *E = out[0];
  if (norm2) *norm2 = out[1];
  return QFD_OK;
}
