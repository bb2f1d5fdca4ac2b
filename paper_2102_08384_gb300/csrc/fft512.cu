// Native FP32 3D FFTs of 512^3 meshes in the library's padded in-place layout.
//
// A 3D real transform is done in two passes over HBM instead of three:
//   plane pass  (one x-plane per 8-CTA thread-block cluster): R2C along z of the
//               plane's 512 rows, then C2C along y of its 257 kz columns, the
//               plane held in the cluster's distributed shared memory;
//   x pass      (tiles of 16 kz columns of one ky): C2C along x.
// The inverse runs the x pass then the mirrored plane pass (C2C along y, C2R
// along z).  The x pass can also apply, between a forward and an inverse
// transform, the spectral product F conj(D) s W^-2 of the convolution steps
// (eq. g-JM-form, eq. 2pcf-yama), so a field goes forward, is multiplied and
// comes back in one read and one write.
//
// 512-point transforms are computed by groups of 64 threads as 8 x 8 x 8
// (three radix-8 stages in registers, two exchanges through shared memory,
// twiddles from a shared FP32 table of exp(-2 pi i j / 512) evaluated in FP64
// on the host).  Real rows are transformed two at a time as the real and
// imaginary parts of one complex sequence.  Transforms are unnormalised, with
// the e^{-i k.x} sign for the forward direction, like cuFFT's.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fft512.h"

namespace cg = cooperative_groups;

namespace bym {
namespace {

constexpr int NM = 512;                  // mesh size handled natively
constexpr int HZ = NM / 2 + 1;           // 257 kz values
constexpr long long ROWF = NM + 2;       // padded real row (floats)
constexpr int CL = 8;                    // CTAs per cluster (one x-plane)
constexpr int ROWS = NM / CL;            // 64 rows per CTA
constexpr int NG = 16;                   // 64-thread groups per CTA (1024 threads)
constexpr int COLS = 32;                 // kz columns owned per CTA (the last owns 33)
constexpr int CPAD = 33;                 // padded column count in the inverse column buffer

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }   // a * i

// In-register forward 8-point DFT, natural order in and out:
// decimation in frequency with radix-2 butterflies, then bit reversal.
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  const float r = 0.70710678118654752f;
  float2 a[8];
  a[0] = cadd(v[0], v[4]);
  a[1] = cadd(v[1], v[5]);
  a[2] = cadd(v[2], v[6]);
  a[3] = cadd(v[3], v[7]);
  a[4] = csub(v[0], v[4]);
  float2 t = csub(v[1], v[5]);
  a[5] = make_float2((t.x + t.y) * r, (t.y - t.x) * r);      // * W8^1 = (1 - i)/sqrt2
  a[6] = mul_mi(csub(v[2], v[6]));                            // * W8^2 = -i
  t = csub(v[3], v[7]);
  a[7] = make_float2((t.y - t.x) * r, -(t.x + t.y) * r);      // * W8^3 = -(1 + i)/sqrt2
  float2 b[8];
  b[0] = cadd(a[0], a[2]);
  b[1] = cadd(a[1], a[3]);
  b[2] = csub(a[0], a[2]);
  b[3] = mul_mi(csub(a[1], a[3]));
  b[4] = cadd(a[4], a[6]);
  b[5] = cadd(a[5], a[7]);
  b[6] = csub(a[4], a[6]);
  b[7] = mul_mi(csub(a[5], a[7]));
  v[0] = cadd(b[0], b[1]);
  v[4] = csub(b[0], b[1]);
  v[2] = cadd(b[2], b[3]);
  v[6] = csub(b[2], b[3]);
  v[1] = cadd(b[4], b[5]);
  v[5] = csub(b[4], b[5]);
  v[3] = cadd(b[6], b[7]);
  v[7] = csub(b[6], b[7]);
}

// Forward 512-point DFT of the sequence held by a 64-thread group:
// on entry thread t holds x[64 n1 + t] in v[n1]; on exit thread t = 8 k1 + j1
// holds X[k1 + 8 j1 + 64 j2] in v[j2].  buf(e) addresses 512 scratch elements
// of this group; sync() synchronises every thread that shares the scratch.
template <class Buf, class Sync>
__device__ __forceinline__ void fft512_group(float2 (&v)[8], int t, const float2 *__restrict__ tw, Buf buf,
                                             Sync sync) {
  // n = 64 n1 + n2 (n2 = t), k = k1 + 8 k2: 8-point DFTs over n1, twiddle W512^(n2 k1)
  dft8(v);
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    v[k1] = cmul(v[k1], tw[(t * k1) & 511]);
    buf(k1 * 64 + t) = v[k1];
  }
  sync();
  // 64-point DFTs over n2 = 8 m1 + m2 for each k1, k2 = j1 + 8 j2
  const int k1 = t >> 3, m2 = t & 7;
#pragma unroll
  for (int m1 = 0; m1 < 8; ++m1) v[m1] = buf(k1 * 64 + 8 * m1 + m2);
  sync();
  dft8(v);
#pragma unroll
  for (int j1 = 0; j1 < 8; ++j1) {
    v[j1] = cmul(v[j1], tw[(8 * m2 * j1) & 511]);
    buf(k1 * 64 + 8 * j1 + m2) = v[j1];
  }
  sync();
  const int j1 = t & 7;
#pragma unroll
  for (int mm = 0; mm < 8; ++mm) v[mm] = buf(k1 * 64 + 8 * j1 + mm);
  sync();
  dft8(v);
}

__device__ __forceinline__ int out_index(int t, int j2) { return (t >> 3) + 8 * (t & 7) + 64 * j2; }

__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ gtw) {
  for (int i = threadIdx.x; i < 512; i += blockDim.x) tw[i] = gtw[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// plane pass, forward: R2C along z, C2C along y, one x-plane per cluster
// grid (8, 512, nslots), block 1024, cluster (8, 1, 1)
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(1024, 1)
    fft512_plane_fwd(float *__restrict__ data, long long slot_reals, const float2 *__restrict__ gtw) {
  extern __shared__ float4 smem4[];
  float2 *tw = (float2 *)smem4;                // 512
  float2 *S = tw + 512;                        // [ROWS][HZ] row spectra of this CTA
  float2 *W = S + ROWS * HZ;                   // [NG][512] scratch, later [512][NG] staging
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int x = blockIdx.y;
  float *plane = data + (long long)blockIdx.z * slot_reals + (long long)x * NM * ROWF;
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  load_twiddles(tw, gtw);
  float2 *Wg = W + g * 512;
  auto bufg = [&](int e) -> float2 & { return Wg[e]; };
  auto sync = [] { __syncthreads(); };
  // R2C along z: 32 row pairs, 16 at a time
#pragma unroll 1
  for (int it = 0; it < ROWS / 2 / NG; ++it) {
    const int p = it * NG + g;
    const int ya = r * ROWS + 2 * p;
    const float *ra = plane + (long long)ya * ROWF, *rb = ra + ROWF;
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = make_float2(ra[64 * n1 + t], rb[64 * n1 + t]);
    fft512_group(v, t, tw, bufg, sync);
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) Wg[out_index(t, j2)] = v[j2];
    __syncthreads();
    // unpack the two real rows: Xa = (Z_k + conj Z_-k)/2, Xb = (Z_k - conj Z_-k)/(2i)
    float2 *Sa = S + (2 * p) * HZ, *Sb = Sa + HZ;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int k = t + 64 * q;
      if (k > 256) break;
      const float2 zk = Wg[k], zm = cconj(Wg[(512 - k) & 511]);
      Sa[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      const float2 d = csub(zk, zm);
      Sb[k] = make_float2(0.5f * d.y, -0.5f * d.x);
    }
    __syncthreads();
  }
  cluster.sync();
  // C2C along y for this CTA's kz columns, 16 at a time (one per group)
  const int c0 = r * COLS, c1 = (r == CL - 1) ? HZ : c0 + COLS;
  float2 *plane_c = (float2 *)plane;
#pragma unroll 1
  for (int base = c0; base < c1; base += NG) {
    const int kz = base + g;
    float2 v[8];
    if (kz < c1) {
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) {
        const float2 *Sr = cluster.map_shared_rank(S, n1);
        v[n1] = Sr[t * HZ + kz];
      }
    } else {
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) v[n1] = make_float2(0.f, 0.f);
    }
    fft512_group(v, t, tw, bufg, sync);
    __syncthreads();
    // stage [ky][g] and write 16 consecutive kz per ky row
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) W[out_index(t, j2) * NG + g] = v[j2];
    __syncthreads();
    for (int i = threadIdx.x; i < 512 * NG; i += blockDim.x) {
      const int ky = i / NG, gg = i % NG;
      if (base + gg < c1) plane_c[(long long)ky * HZ + base + gg] = W[i];
    }
    __syncthreads();
  }
  cluster.sync();
}

// ---------------------------------------------------------------------------
// plane pass, inverse: C2C along y (inverse), C2R along z
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(1024, 1)
    fft512_plane_inv(float *__restrict__ data, long long slot_reals, const float2 *__restrict__ gtw) {
  extern __shared__ float4 smem4[];
  float2 *tw = (float2 *)smem4;                // 512
  float2 *Tc = tw + 512;                       // [512][CPAD] y-transformed columns of this CTA
  float2 *W = Tc + 512 * CPAD;                 // [512][NG] staging / [NG][512] scratch
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int x = blockIdx.y;
  float *plane = data + (long long)blockIdx.z * slot_reals + (long long)x * NM * ROWF;
  const float2 *plane_c = (const float2 *)plane;
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  load_twiddles(tw, gtw);
  float2 *Wg = W + g * 512;
  auto bufg = [&](int e) -> float2 & { return Wg[e]; };
  auto sync = [] { __syncthreads(); };
  const int c0 = r * COLS, c1 = (r == CL - 1) ? HZ : c0 + COLS;
#pragma unroll 1
  for (int base = c0; base < c1; base += NG) {
    for (int i = threadIdx.x; i < 512 * NG; i += blockDim.x) {
      const int ky = i / NG, gg = i % NG;
      W[i] = (base + gg < c1) ? plane_c[(long long)ky * HZ + base + gg] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = cconj(W[(64 * n1 + t) * NG + g]);   // inverse via conjugation
    __syncthreads();
    fft512_group(v, t, tw, bufg, sync);
    const int kl = base - c0 + g;
    if (base + g < c1) {
#pragma unroll
      for (int j2 = 0; j2 < 8; ++j2) Tc[out_index(t, j2) * CPAD + kl] = cconj(v[j2]);
    }
    __syncthreads();
  }
  cluster.sync();
  // C2R along z: two rows at a time as Z = Xa + i Xb, Hermitian-extended to 512
#pragma unroll 1
  for (int it = 0; it < ROWS / 2 / NG; ++it) {
    const int p = it * NG + g;
    const int ya = r * ROWS + 2 * p, yb = ya + 1;
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      const int k = 64 * n1 + t;
      const int kk = k <= 256 ? k : 512 - k;
      const int own = kk / COLS < CL ? kk / COLS : CL - 1;
      const float2 *To = cluster.map_shared_rank(Tc, min(own, CL - 1));
      const int kl = kk - own * COLS;
      float2 xa = To[ya * CPAD + kl], xb = To[yb * CPAD + kl];
      if (k > 256) {
        xa = cconj(xa);
        xb = cconj(xb);
      }
      v[n1] = cconj(cadd(xa, mul_i(xb)));      // inverse via conjugation
    }
    fft512_group(v, t, tw, bufg, sync);
    float *ra = plane + (long long)ya * ROWF, *rb = plane + (long long)yb * ROWF;
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) {
      const int k = out_index(t, j2);
      const float2 z = cconj(v[j2]);
      ra[k] = z.x;
      rb[k] = z.y;
    }
    __syncthreads();
  }
  cluster.sync();
}

// ---------------------------------------------------------------------------
// x pass: C2C along x for tiles of 16 kz columns of one ky
// mode 0 forward, 1 inverse, 2 forward -> * conj(D) s_f W^-2 -> inverse
// grid (17, 512, nslots), block 1024 (g = tid % 16 the column, t = tid / 16)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(1024, 1)
    fft512_x(float2 *__restrict__ data, long long slot_cplx, const float2 *__restrict__ gtw,
             const float2 *__restrict__ D, const double *__restrict__ scale, const float *__restrict__ invw) {
  extern __shared__ float4 smem4[];
  float2 *tw = (float2 *)smem4;   // 512
  float2 *W = tw + 512;           // [512][16]
  const int g = threadIdx.x & 15, t = threadIdx.x >> 4;
  const int kz = blockIdx.x * 16 + g, ky = blockIdx.y;
  const bool valid = kz < HZ;
  float2 *col = data + (long long)blockIdx.z * slot_cplx + (long long)ky * HZ + kz;
  const long long xs = (long long)NM * HZ;    // stride between consecutive x
  load_twiddles(tw, gtw);
  auto buf = [&](int e) -> float2 & { return W[e * 16 + g]; };
  auto sync = [] { __syncthreads(); };
  float2 v[8];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) {
    const float2 a = valid ? col[(64 * n1 + t) * xs] : make_float2(0.f, 0.f);
    v[n1] = MODE == 1 ? cconj(a) : a;
  }
  fft512_group(v, t, tw, buf, sync);
  if (MODE == 2) {
    const float s = (float)scale[blockIdx.z];
    float cyz = 1.f;
    if (invw) cyz = invw[ky] * invw[valid ? kz : 0];
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) {
      const int kx = out_index(t, j2);
      float2 d = valid ? D[(long long)kx * xs + (long long)ky * HZ + kz] : make_float2(0.f, 0.f);
      float c = s;
      if (invw) {
        const float cc = invw[kx] * cyz;
        c *= cc * cc;
      }
      const float2 p = cmul(v[j2], cconj(d));
      v[j2] = make_float2(p.x * c, p.y * c);
    }
    __syncthreads();
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) W[out_index(t, j2) * 16 + g] = v[j2];
    __syncthreads();
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = cconj(W[(64 * n1 + t) * 16 + g]);
    __syncthreads();
    fft512_group(v, t, tw, buf, sync);
  }
  if (valid) {
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) {
      const float2 o = (MODE == 0) ? v[j2] : cconj(v[j2]);
      col[(long long)out_index(t, j2) * xs] = o;
    }
  }
}

float2 *g_twiddles[64] = {nullptr};
std::mutex g_tw_mu;

const float2 *twiddles(int dev) {
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (!g_twiddles[dev]) {
    float2 host[512];
    for (int j = 0; j < 512; ++j) {
      const double a = -2.0 * M_PI * j / 512.0;
      host[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    float2 *d = nullptr;
    if (cudaMalloc(&d, sizeof host) != cudaSuccess) return nullptr;
    cudaMemcpy(d, host, sizeof host, cudaMemcpyHostToDevice);
    g_twiddles[dev] = d;
  }
  return g_twiddles[dev];
}

constexpr size_t kPlaneFwdSmem = sizeof(float2) * (512 + ROWS * HZ + NG * 512);
constexpr size_t kPlaneInvSmem = sizeof(float2) * (512 + 512 * CPAD + NG * 512);
constexpr size_t kXSmem = sizeof(float2) * (512 + 512 * 16);

}  // namespace

bool native_fft_supported(int n_mesh, int precision) { return n_mesh == NM && precision == 32; }

cudaError_t native_fft_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!twiddles(dev)) return cudaErrorMemoryAllocation;
  static bool attrs[64] = {false};
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (!attrs[dev]) {
    if ((e = cudaFuncSetAttribute(fft512_plane_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPlaneFwdSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_plane_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPlaneInvSmem)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_x<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXSmem)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_x<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXSmem)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_x<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXSmem)) !=
        cudaSuccess)
      return e;
    attrs[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t native_fft_forward(float *slots, long long slot_reals, int first, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  for (int done = 0; done < count; done += 65535) {
    const int n = count - done < 65535 ? count - done : 65535;
    float *b = base + (long long)done * slot_reals;
    fft512_plane_fwd<<<dim3(CL, NM, n), 1024, kPlaneFwdSmem, st>>>(b, slot_reals, tw);
    fft512_x<0><<<dim3((HZ + 15) / 16, NM, n), 1024, kXSmem, st>>>((float2 *)b, slot_reals / 2, tw, nullptr,
                                                                   nullptr, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t native_fft_inverse(float *slots, long long slot_reals, int first, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  for (int done = 0; done < count; done += 65535) {
    const int n = count - done < 65535 ? count - done : 65535;
    float *b = base + (long long)done * slot_reals;
    fft512_x<1><<<dim3((HZ + 15) / 16, NM, n), 1024, kXSmem, st>>>((float2 *)b, slot_reals / 2, tw, nullptr,
                                                                   nullptr, nullptr);
    fft512_plane_inv<<<dim3(CL, NM, n), 1024, kPlaneInvSmem, st>>>(b, slot_reals, tw);
  }
  return cudaGetLastError();
}

cudaError_t native_fft_convolve(float *slots, long long slot_reals, int first, int count, const float *D,
                                const double *scale, const float *invw, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  for (int done = 0; done < count; done += 65535) {
    const int n = count - done < 65535 ? count - done : 65535;
    float *b = base + (long long)done * slot_reals;
    fft512_plane_fwd<<<dim3(CL, NM, n), 1024, kPlaneFwdSmem, st>>>(b, slot_reals, tw);
    fft512_x<2><<<dim3((HZ + 15) / 16, NM, n), 1024, kXSmem, st>>>((float2 *)b, slot_reals / 2, tw,
                                                                   (const float2 *)D, scale + done, invw);
    fft512_plane_inv<<<dim3(CL, NM, n), 1024, kPlaneInvSmem, st>>>(b, slot_reals, tw);
  }
  return cudaGetLastError();
}

}  // namespace bym
