// Yamamoto k-space contraction for callers that cannot allocate device memory.
//
// Some host applications cannot call cudaMalloc at the point where they want
// multipoles: an allocator owned by another framework that must not be
// bypassed, a fixed memory budget carved out before the run, or code that
// runs while allocation is forbidden.  bym_pk_yamamoto_from_spectra_noalloc
// serves them: the caller passes the field spectra it already holds and host
// output arrays, and every piece of scratch (bin table, FP64 shell sums, mode
// counts, the bin edges) lives in one file-scope __device__ array of
// kScratchBytes that each GPU loading the library holds until the process
// exits.  No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "bym.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxBins = 1024;
constexpr int kMaxMesh = 512;
constexpr int kMaxEllMax = 4;
constexpr int kNL = kMaxEllMax / 2 + 1;
constexpr long long kLutLen = 3LL * (kMaxMesh / 2) * (kMaxMesh / 2) + 1;
// scratch layout (bytes): edges | sums [kNL][kMaxBins] | counts [kMaxBins] | lut [kLutLen]
constexpr size_t kOffEdges = 0;
constexpr size_t kOffSums = 8448;
constexpr size_t kOffCounts = kOffSums + sizeof(double) * kNL * kMaxBins;
constexpr size_t kOffLut = kOffCounts + sizeof(unsigned long long) * kMaxBins;
constexpr size_t kScratchBytes = 1u << 20;  // 1 MiB
static_assert(kOffLut + sizeof(int) * kLutLen <= kScratchBytes, "scratch layout exceeds its array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};
int g_nsm[kMaxDevices] = {0};

// Device address of the scratch array and the device's SM count, looked up once per device
// with that device current (in host code the symbol itself is only a host-side handle).
cudaError_t scratch_address(int dev, unsigned char **out, int *nsm) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    g_nsm[dev] = n > 0 ? n : 1;
    g_addr[dev] = p;
  }
  *out = (unsigned char *)g_addr[dev];
  *nsm = g_nsm[dev];
  return cudaSuccess;
}

__host__ __device__ constexpr double csqrt(double x) {
  double r = x > 1.0 ? x : 1.0;
  for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
  return r;
}

// Recurrence constants of the real spherical harmonics up to l = 4, evaluated
// at compile time into constant memory.
struct YlmTab {
  float mm[5];     // normalised P_mm
  float first[5];  // P_{m+1,m} = first[m] z P_mm
  float a[5][5], b[5][5];
};

constexpr YlmTab make_ylm_tab() {
  YlmTab t{};
  double pmm = 1.0 / csqrt(4.0 * 3.14159265358979323846);
  for (int m = 0; m <= 4; ++m) {
    if (m > 0) pmm *= csqrt((2.0 * m + 1) / (2.0 * m));
    t.mm[m] = (float)pmm;
    t.first[m] = (float)csqrt(2.0 * m + 3);
    for (int l = m + 2; l <= 4; ++l) {
      t.a[l][m] = (float)csqrt((4.0 * l * l - 1) / ((double)l * l - (double)m * m));
      t.b[l][m] = (float)csqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1));
    }
  }
  return t;
}

__constant__ YlmTab kYlm = make_ylm_tab();

// Real spherical harmonics, l <= 4, by the associated-Legendre recurrence
// (orthonormal, no Condon-Shortley phase): Y[l*l + l + m].
__device__ __forceinline__ void real_ylm4(float x, float y, float z, float (&Y)[25]) {
  float c[5], s[5];
  c[0] = 1.f;
  s[0] = 0.f;
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    c[m] = c[m - 1] * x - s[m - 1] * y;
    s[m] = s[m - 1] * x + c[m - 1] * y;
  }
#pragma unroll
  for (int m = 0; m <= 4; ++m) {
    float p2 = 0.f, p1 = kYlm.mm[m];
#pragma unroll
    for (int l = m; l <= 4; ++l) {
      float p;
      if (l == m) {
        p = kYlm.mm[m];
      } else if (l == m + 1) {
        p = kYlm.first[m] * z * p1;
      } else {
        p = kYlm.a[l][m] * (z * p1 - kYlm.b[l][m] * p2);
      }
      if (l > m) {
        p2 = p1;
        p1 = p;
      }
      if (m == 0) {
        Y[l * l + l] = p;
      } else {
        Y[l * l + l + m] = 1.41421356237309515f * p * c[m];
        Y[l * l + l - m] = 1.41421356237309515f * p * s[m];
      }
    }
  }
}

__global__ void noalloc_setup(int N, int nbins, double kf, unsigned char *scratch) {
  const double *edges = (const double *)(scratch + kOffEdges);
  double *sums = (double *)(scratch + kOffSums);
  unsigned long long *counts = (unsigned long long *)(scratch + kOffCounts);
  int *lut = (int *)(scratch + kOffLut);
  const long long n2max = 3LL * (N / 2) * (N / 2);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n2max; i += stride) {
    int bin = -1;
    if (i > 0) {
      const double mag = kf * sqrt((double)i);
      int lo = 0, hi = nbins + 1;        // first edge > mag (upper bound), then step back
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (edges[mid] > mag)
          hi = mid;
        else
          lo = mid + 1;
      }
      bin = lo - 1;
      if (bin >= nbins) bin = -1;
    }
    lut[i] = bin;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)kNL * kMaxBins; i += stride)
    sums[i] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < kMaxBins; i += stride) counts[i] = 0ULL;
}

// P_l sums of the Yamamoto estimator: sum over half-spectrum modes of
// w(k) sum_mu Y_{l mu}(hat k) Re[F_{l mu}(k) conj(D(k))], w = 1 on the kz = 0
// and Nyquist planes and 2 elsewhere; FP64 accumulation.
template <int NL>
__global__ void __launch_bounds__(256) noalloc_contract(const float2 *__restrict__ F, const float2 *__restrict__ D,
                                                        int N, int nbins, unsigned char *scratch) {
  double *sums = (double *)(scratch + kOffSums);
  unsigned long long *counts = (unsigned long long *)(scratch + kOffCounts);
  const int *lut = (const int *)(scratch + kOffLut);
  __shared__ double ssum[NL][kMaxBins];
  __shared__ unsigned long long scnt[kMaxBins];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
#pragma unroll
    for (int l = 0; l < NL; ++l) ssum[l][i] = 0.0;
    scnt[i] = 0ULL;
  }
  __syncthreads();
  const int H = N / 2 + 1;
  const long long nm = (long long)N * N * H;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(m % H);
    const long long row = m / H;
    const int ix = (int)(row / N), iy = (int)(row % N);
    const int nx = ix < N / 2 ? ix : ix - N, ny = iy < N / 2 ? iy : iy - N, nz = (iz == N / 2) ? -N / 2 : iz;
    const int n2 = nx * nx + ny * ny + nz * nz;
    const int bin = lut[n2];
    if (bin < 0) continue;
    const float ir = rsqrtf((float)n2);
    float Y[25];
    real_ylm4(nx * ir, ny * ir, nz * ir, Y);
    const float2 d = D[m];
    const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;
    int f = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int ell = 2 * l;
      float T = 0.f;
#pragma unroll
      for (int mu = -ell; mu <= ell; ++mu, ++f) {
        const float2 a = F[(long long)f * nm + m];
        T += Y[ell * ell + ell + mu] * (a.x * d.x + a.y * d.y);
      }
      atomicAdd(&ssum[l][bin], w * (double)T);
    }
    atomicAdd(&scnt[bin], (unsigned long long)w);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
#pragma unroll
    for (int l = 0; l < NL; ++l)
      if (ssum[l][i] != 0.0) atomicAdd(sums + l * kMaxBins + i, ssum[l][i]);
    if (scnt[i]) atomicAdd(counts + i, scnt[i]);
  }
}

}  // namespace

extern "C" int bym_pk_yamamoto_from_spectra_noalloc(const void *F, const void *D, int n_mesh, double box_len,
                                                    int ell_max, const bym_bins *kbins, double norm_A, double *pk,
                                                    int64_t *n_modes, void *cuda_stream) {
  if (!F || !D || !kbins || !kbins->edges || !pk || !n_modes) return BYM_E_INVAL;
  if (n_mesh < 8 || n_mesh % 2) return BYM_E_INVAL;
  if (n_mesh > kMaxMesh) return BYM_E_UNSUPPORTED;          // bin table would not fit the scratch array
  if (ell_max < 0 || ell_max % 2 || ell_max > kMaxEllMax) return BYM_E_UNSUPPORTED;
  if (kbins->nbins < 1 || kbins->nbins > kMaxBins) return BYM_E_UNSUPPORTED;
  if (!(box_len > 0.0) || !(norm_A > 0.0)) return BYM_E_INVAL;
  for (int i = 0; i < kbins->nbins; ++i)
    if (!(kbins->edges[i + 1] > kbins->edges[i]) || !std::isfinite(kbins->edges[i + 1])) return BYM_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BYM_E_CUDA;
  unsigned char *scratch = nullptr;
  int nsm = 1;
  if (scratch_address(dev, &scratch, &nsm) != cudaSuccess) return BYM_E_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int N = n_mesh, nb = kbins->nbins, NL = ell_max / 2 + 1;
  if (cudaMemcpyAsync(scratch + kOffEdges, kbins->edges, sizeof(double) * (nb + 1), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return BYM_E_CUDA;
  const double kf = 2.0 * M_PI / box_len;
  noalloc_setup<<<256, 256, 0, st>>>(N, nb, kf, scratch);
  const long long nm = (long long)N * N * (N / 2 + 1);
  const unsigned grid = (unsigned)std::min<long long>((nm + 255) / 256, (long long)nsm * 8);
  const float2 *Fp = (const float2 *)F, *Dp = (const float2 *)D;
  if (NL == 1)
    noalloc_contract<1><<<grid, 256, 0, st>>>(Fp, Dp, N, nb, scratch);
  else if (NL == 2)
    noalloc_contract<2><<<grid, 256, 0, st>>>(Fp, Dp, N, nb, scratch);
  else
    noalloc_contract<3><<<grid, 256, 0, st>>>(Fp, Dp, N, nb, scratch);
  if (cudaGetLastError() != cudaSuccess) return BYM_E_CUDA;
  // copy the FP64 sums [l][bin] straight into pk and the counts into n_modes
  for (int l = 0; l < NL; ++l)
    if (cudaMemcpyAsync(pk + (size_t)l * nb, scratch + kOffSums + sizeof(double) * l * kMaxBins,
                        sizeof(double) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return BYM_E_CUDA;
  static_assert(sizeof(int64_t) == sizeof(unsigned long long), "count width");
  if (cudaMemcpyAsync(n_modes, scratch + kOffCounts, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BYM_E_CUDA;
  const double four_pi = 4.0 * M_PI;
  for (int l = 0; l < NL; ++l)
    for (int b = 0; b < nb; ++b) {
      double &v = pk[(size_t)l * nb + b];
      v = n_modes[b] > 0 ? four_pi / norm_A * v / (double)n_modes[b] : 0.0;
    }
  return BYM_OK;
}
