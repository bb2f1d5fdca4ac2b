// Native FP32 3D FFTs of 512^3 meshes in the library's padded in-place layout.
//
// A 3D real transform is done in two passes over HBM instead of three:
//   plane pass  (one x-plane per thread-block cluster of CL CTAs): R2C along z of
//               the plane's 512 rows, then C2C along y of its 257 kz columns;
//               each CTA owns 512/CL rows and 256/CL columns, and the row
//               spectra go straight to the owner of each column by stores into
//               its distributed shared memory;
//   x pass      (tiles of 16 consecutive (ky, kz) columns, moved by TMA): C2C along x.
// The inverse runs the x pass then the mirrored plane pass (C2C along y, C2R
// along z).  The x pass can also apply, between a forward and an inverse
// transform, the spectral product F conj(D) s W^-2 of the convolution steps
// (eq. g-JM-form, eq. 2pcf-yama), so a field goes forward, is multiplied and
// comes back in one read and one write.
//
// Every 512-point transform is computed by a group of 16 threads holding 32
// values each, as 512 = 32 x 16: a 32-point DFT in registers, twiddles
// W512^(j k1), one exchange through a padded (bank-conflict-free) shared
// buffer, and 16-point DFTs in registers.  Thread j of a group starts with
// x[16 m + j] (m = 0..31) and ends with X[ka + 32 k2] and X[kb + 32 k2]
// (k2 = 0..15) for the column pair ka = j, kb = 32 - j (kb = 16 for j = 0), so
// that X[k] and X[512 - k] always sit in the same thread: the packing of two
// real sequences into one complex transform is undone in registers.  The
// inverse runs the same steps backwards from that layout.  The kz = 0 and
// kz = 256 columns of a plane, real sequences along y, share one complex
// column transform.  Transforms are unnormalised, with the e^{-i k.x} sign for
// the forward direction, like cuFFT's.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "fft512.h"

namespace cg = cooperative_groups;

namespace bym {
namespace {

constexpr int NM = 512;                  // mesh size handled natively
constexpr int HP = NM / 2 + 2;           // complex pitch of a row: 258 (the last value is padding)
constexpr long long ROWF = 2 * HP;       // padded real row (floats): 2064 bytes, 16-byte aligned
constexpr int CS = 514;                  // column stride (float2) of the column buffer; even for float4 pairs
constexpr int ES = 17;                   // row stride (float2) of the exchange buffer and twiddle table
constexpr int EX = 32 * ES;              // exchange buffer of one group (float2)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// cos(pi p / 16), p = 0..8
__device__ __forceinline__ float cos_pi16(int p) {
  switch (p) {
    case 0: return 1.0f;
    case 1: return 0.98078528040323044913f;
    case 2: return 0.92387953251128675613f;
    case 3: return 0.83146961230254523708f;
    case 4: return 0.70710678118654752440f;
    case 5: return 0.55557023301960222474f;
    case 6: return 0.38268343236508977173f;
    case 7: return 0.19509032201612826785f;
    default: return 0.0f;
  }
}

// a * exp(-2 pi i p / 32), p = 0..15 (a compile-time constant after unrolling)
__device__ __forceinline__ float2 w32mul(float2 a, int p) {
  if (p == 0) return a;
  if (p == 8) return make_float2(a.y, -a.x);
  const float c = p < 8 ? cos_pi16(p) : -cos_pi16(16 - p);
  const float s = p < 8 ? cos_pi16(8 - p) : cos_pi16(p - 8);
  return make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <int BITS>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 0; b < BITS; ++b) r |= ((k >> b) & 1) << (BITS - 1 - b);
  return r;
}

// In-register forward DFT of L = 2^LOG points (L <= 32), natural order in and out:
// radix-2 decimation in frequency, then the bit-reversal permutation (a renaming).
template <int L, int LOG>
__device__ __forceinline__ void dft(float2 (&v)[L]) {
#pragma unroll
  for (int s = 0; s < LOG; ++s) {
    const int h = L >> (s + 1);
#pragma unroll
    for (int b = 0; b < L; b += 2 * h) {
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const float2 a = v[b + i], c = v[b + i + h];
        v[b + i] = cadd(a, c);
        v[b + i + h] = w32mul(csub(a, c), i * (32 / (2 * h)));
      }
    }
  }
  float2 t[L];
#pragma unroll
  for (int k = 0; k < L; ++k) t[k] = v[bitrev<LOG>(k)];
#pragma unroll
  for (int k = 0; k < L; ++k) v[k] = t[k];
}

template <int L, int LOG>
__device__ __forceinline__ void idft(float2 (&v)[L]) {  // e^{+i} direction, unnormalised
#pragma unroll
  for (int k = 0; k < L; ++k) v[k] = cconj(v[k]);
  dft<L, LOG>(v);
#pragma unroll
  for (int k = 0; k < L; ++k) v[k] = cconj(v[k]);
}

__device__ __forceinline__ int col_b(int j) { return j ? 32 - j : 16; }

// Twiddles of thread j of a group: fwd(k1) = W512^(k1 j), k1 = 1..31; inv_a(n1) = W512^(ka n1),
// inv_b(n1) = W512^(kb n1), n1 = 1..15 (ka = j, kb = col_b(j)).  TabTw reads them from the padded
// shared table TW[k1 * ES + j] = W512^(k1 j).
struct TabTw {
  const float2 *TW;
  int j, kb;
  __device__ __forceinline__ float2 fwd(int k1) const { return TW[k1 * ES + j]; }
  __device__ __forceinline__ float2 inv_a(int n1) const { return TW[j * ES + n1]; }
  __device__ __forceinline__ float2 inv_b(int n1) const { return TW[kb * ES + n1]; }
};

// Exchange storage of a 16-thread group, 32 x 16 complex slots (a, b): a padded row-major
// buffer (row stride ES, bank-conflict free).
struct PadEx {
  float2 *E;
  __device__ __forceinline__ float2 &operator()(int a, int b) const { return E[a * ES + b]; }
};

// Forward 512-point DFT by a 16-thread group.  In: v[m] = x[16 m + j].
// Out: A[k2] = X[ka + 32 k2], B[k2] = X[kb + 32 k2].  TW[k1 * ES + j] = W512^(k1 j);
// ex: this group's exchange storage, slots (a, b) with a < 32, b < 16 (a < 16 with HALF: the
// exchange then runs in two rounds, k1 < 16 then k1 >= 16); gm: this group's lane mask.
template <bool HALF = false, class EXS, class TWS>
__device__ __forceinline__ void fwd512x(float2 (&v)[32], float2 (&A)[16], float2 (&B)[16], int j, unsigned gm,
                                       const TWS &tw, const EXS &ex) {
  dft<32, 5>(v);
#pragma unroll
  for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], tw.fwd(k1));
  const int ka = j, kb = col_b(j);
  __syncwarp(gm);
  if (HALF) {
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) ex(k1, j) = v[k1];
    __syncwarp(gm);
#pragma unroll
    for (int i = 0; i < 16; ++i) A[i] = ex(ka, i);
    __syncwarp(gm);
#pragma unroll
    for (int k1 = 16; k1 < 32; ++k1) ex(k1 - 16, j) = v[k1];
    __syncwarp(gm);
#pragma unroll
    for (int i = 0; i < 16; ++i) B[i] = ex(kb - 16, i);
  } else {
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) ex(k1, j) = v[k1];
    __syncwarp(gm);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      A[i] = ex(ka, i);
      B[i] = ex(kb, i);
    }
  }
  dft<16, 4>(A);
  dft<16, 4>(B);
}

template <bool HALF = false>
__device__ __forceinline__ void fwd512(float2 (&v)[32], float2 (&A)[16], float2 (&B)[16], int j, unsigned gm,
                                       const float2 *__restrict__ TW, float2 *E) {
  fwd512x<HALF>(v, A, B, j, gm, TabTw{TW, j, col_b(j)}, PadEx{E});
}

// Inverse (e^{+i}, unnormalised) 512-point DFT by a 16-thread group, from the
// layout fwd512 produces to v[m] = x[16 m + j].
template <bool HALF = false, class EXS, class TWS>
__device__ __forceinline__ void inv512x(float2 (&A)[16], float2 (&B)[16], float2 (&v)[32], int j, unsigned gm,
                                       const TWS &tw, const EXS &ex) {
  idft<16, 4>(A);
  idft<16, 4>(B);
  const int ka = j, kb = col_b(j);
#pragma unroll
  for (int n1 = 1; n1 < 16; ++n1) {
    A[n1] = cmulc(A[n1], tw.inv_a(n1));
    B[n1] = cmulc(B[n1], tw.inv_b(n1));
  }
  __syncwarp(gm);
  if (HALF) {
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) ex(ka, n1) = A[n1];
    __syncwarp(gm);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = ex(k1, j);
    __syncwarp(gm);
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) ex(kb - 16, n1) = B[n1];
    __syncwarp(gm);
#pragma unroll
    for (int k1 = 16; k1 < 32; ++k1) v[k1] = ex(k1 - 16, j);
  } else {
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
      ex(ka, n1) = A[n1];
      ex(kb, n1) = B[n1];
    }
    __syncwarp(gm);
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) v[k1] = ex(k1, j);
  }
  idft<32, 5>(v);
}

template <bool HALF = false>
__device__ __forceinline__ void inv512(float2 (&A)[16], float2 (&B)[16], float2 (&v)[32], int j, unsigned gm,
                                       const float2 *__restrict__ TW, float2 *E) {
  inv512x<HALF>(A, B, v, j, gm, TabTw{TW, j, col_b(j)}, PadEx{E});
}

// Two spectra from the transform of z = a + i b (a, b real sequences):
// (A_k, B_k) = ((z_k + conj z_-k) / 2, (z_k - conj z_-k) / 2i); zm = conj z_-k.
__device__ __forceinline__ float4 unpack2(float2 z, float2 zm) {
  const float2 d = csub(z, zm);
  return make_float4(0.5f * (z.x + zm.x), 0.5f * (z.y + zm.y), 0.5f * d.y, -0.5f * d.x);
}

// z = a + i b for complex a, b
__device__ __forceinline__ float2 pack2(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// CL CTAs per cluster.  8: 256 threads, two row pairs and two columns per group, one
// CTA per SM.  16: 256 threads, one row pair and one column per group, the exchange
// in two rounds, 107 KB of shared memory and at most 128 registers so that two CTAs
// (of different clusters) share an SM and overlap their loads and transforms.
template <int CL>
struct PlaneShape {
  static constexpr int CPR = 256 / CL;          // kz columns per CTA (+ kz = 256 on rank 0)
  static constexpr int RPR = NM / CL;           // rows per CTA
  static constexpr int NG = 16;                 // 16-thread groups per CTA
  static constexpr int NT = NG * 16;            // threads per CTA
  static constexpr int ITER = CPR / NG;         // row pairs (RPR / 2) and columns per group
  static constexpr bool HALF = CL == 16;        // half-size exchange buffers
  static constexpr int EXG = HALF ? EX / 2 : EX;
  static constexpr int MINB = CL == 16 ? 2 : 1; // CTAs per SM the register budget allows
  static constexpr size_t SMEM = sizeof(float2) * (EX + (size_t)(CPR + 1) * CS + (size_t)NG * EXG);
};

// ---------------------------------------------------------------------------
// plane pass, forward: R2C along z, C2C along y; one x-plane per cluster
// grid (CL, 512, nslots), cluster (CL, 1, 1)
// ---------------------------------------------------------------------------
template <int CL>
__global__ void __launch_bounds__(PlaneShape<CL>::NT, PlaneShape<CL>::MINB)
    fft512_plane_fwd(float *__restrict__ data, long long slot_reals, const float2 *__restrict__ gtw) {
  using S = PlaneShape<CL>;
  extern __shared__ float4 smem4[];
  float2 *TW = (float2 *)smem4;                 // [32][ES]
  float2 *C = TW + EX;                          // [CPR + 1][CS] columns of this CTA, all 512 y
  float2 *E = C + (S::CPR + 1) * CS;            // [NG][EX]
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  cluster_arrive_relaxed();                     // every CTA of the cluster runs before remote stores
  float *plane = data + (long long)blockIdx.z * slot_reals + (long long)blockIdx.y * NM * ROWF;
  const int tid = threadIdx.x, g = tid >> 4, j = tid & 15;
  const unsigned gm = 0xFFFFu << (tid & 16);
  const int ka = j, kb = col_b(j);
  float2 *Eg = E + g * S::EXG;
  for (int i = tid; i < EX; i += S::NT) TW[i] = gtw[i];
  __syncthreads();
  // R2C along z, two rows at a time; the row spectra go to the owners of their kz
#pragma unroll 1
  for (int it = 0; it < S::ITER; ++it) {
    const int ya = r * S::RPR + 2 * (it * S::NG + g);
    const float *ra = plane + (long long)ya * ROWF, *rb = ra + ROWF;
    float2 v[32], A[16], B[16];
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = make_float2(ra[16 * m + j], rb[16 * m + j]);
    fwd512<S::HALF>(v, A, B, j, gm, TW, Eg);
    if (it == 0) cluster_wait();
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      float4 va = unpack2(A[k2], j ? cconj(B[15 - k2]) : cconj(A[(16 - k2) & 15]));
      if (j == 0 && k2 == 0) {                  // kz = 0 and kz = 256 (both real) share a column
        va.y = A[8].x;
        va.w = A[8].y;
      }
      const float4 vb = unpack2(B[k2], j ? cconj(A[15 - k2]) : cconj(B[15 - k2]));
      const int kza = ka + 32 * k2, kzb = kb + 32 * k2;
      float2 *Ca = cluster.map_shared_rank(C, kza / S::CPR);
      float2 *Cb = cluster.map_shared_rank(C, kzb / S::CPR);
      *(float4 *)(Ca + (kza % S::CPR) * CS + ya) = va;
      *(float4 *)(Cb + (kzb % S::CPR) * CS + ya) = vb;
    }
  }
  cluster_arrive();
  cluster_wait();
  // C2C along y for this CTA's columns; rank 0's first column holds kz = 0 + i kz = 256
#pragma unroll 1
  for (int it = 0; it < S::ITER; ++it) {
    const int kl = it * S::NG + g;
    float2 *col = C + kl * CS;
    float2 v[32], A[16], B[16];
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = col[16 * m + j];
    fwd512<S::HALF>(v, A, B, j, gm, TW, Eg);
    if (r == 0 && kl == 0) {
      float2 *col256 = C + S::CPR * CS;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const float4 a = unpack2(A[k2], j ? cconj(B[15 - k2]) : cconj(A[(16 - k2) & 15]));
        const float4 b = unpack2(B[k2], j ? cconj(A[15 - k2]) : cconj(B[15 - k2]));
        col[ka + 32 * k2] = make_float2(a.x, a.y);
        col256[ka + 32 * k2] = make_float2(a.z, a.w);
        col[kb + 32 * k2] = make_float2(b.x, b.y);
        col256[kb + 32 * k2] = make_float2(b.z, b.w);
      }
    } else {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        col[ka + 32 * k2] = A[k2];
        col[kb + 32 * k2] = B[k2];
      }
    }
  }
  __syncthreads();
  // coalesced write-out: rows ky, ky + 1 of this CTA's kz range
  float2 *pc = (float2 *)plane;
  for (int e = tid; e < 256 * S::CPR; e += S::NT) {
    const int c = e % S::CPR, ky = 2 * (e / S::CPR);
    const float4 val = *(const float4 *)(C + c * CS + ky);
    pc[(long long)ky * HP + r * S::CPR + c] = make_float2(val.x, val.y);
    pc[(long long)(ky + 1) * HP + r * S::CPR + c] = make_float2(val.z, val.w);
  }
  if (r == 0)
    for (int ky = tid; ky < NM; ky += S::NT) pc[(long long)ky * HP + 256] = C[S::CPR * CS + ky];
}

// ---------------------------------------------------------------------------
// plane pass, inverse: C2C along y (inverse), C2R along z
// ---------------------------------------------------------------------------
template <int CL>
__global__ void __launch_bounds__(PlaneShape<CL>::NT, PlaneShape<CL>::MINB)
    fft512_plane_inv(float *__restrict__ data, long long slot_reals, const float2 *__restrict__ gtw) {
  using S = PlaneShape<CL>;
  extern __shared__ float4 smem4[];
  float2 *TW = (float2 *)smem4;
  float2 *C = TW + EX;
  float2 *E = C + (S::CPR + 1) * CS;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  float *plane = data + (long long)blockIdx.z * slot_reals + (long long)blockIdx.y * NM * ROWF;
  const float2 *pc = (const float2 *)plane;
  const int tid = threadIdx.x, g = tid >> 4, j = tid & 15;
  const unsigned gm = 0xFFFFu << (tid & 16);
  const int ka = j, kb = col_b(j);
  float2 *Eg = E + g * S::EXG;
  for (int i = tid; i < EX; i += S::NT) TW[i] = gtw[i];
  // coalesced read of this CTA's kz range
  for (int e = tid; e < 256 * S::CPR; e += S::NT) {
    const int c = e % S::CPR, ky = 2 * (e / S::CPR);
    const float2 a = pc[(long long)ky * HP + r * S::CPR + c];
    const float2 b = pc[(long long)(ky + 1) * HP + r * S::CPR + c];
    *(float4 *)(C + c * CS + ky) = make_float4(a.x, a.y, b.x, b.y);
  }
  if (r == 0)
    for (int ky = tid; ky < NM; ky += S::NT) C[S::CPR * CS + ky] = pc[(long long)ky * HP + 256];
  __syncthreads();
  // inverse C2C along y; rank 0 transforms kz = 0 + i kz = 256 (both real along y after it)
#pragma unroll 1
  for (int it = 0; it < S::ITER; ++it) {
    const int kl = it * S::NG + g;
    float2 *col = C + kl * CS;
    float2 v[32], A[16], B[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      A[k2] = col[ka + 32 * k2];
      B[k2] = col[kb + 32 * k2];
    }
    if (r == 0 && kl == 0) {
      const float2 *col256 = C + S::CPR * CS;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        A[k2] = pack2(A[k2], col256[ka + 32 * k2]);
        B[k2] = pack2(B[k2], col256[kb + 32 * k2]);
      }
    }
    inv512<S::HALF>(A, B, v, j, gm, TW, Eg);
#pragma unroll
    for (int m = 0; m < 32; ++m) col[16 * m + j] = v[m];
  }
  cluster_arrive();
  cluster_wait();
  // C2R along z, two rows at a time as z = a + i b; the half spectra come from the column owners
#pragma unroll 1
  for (int it = 0; it < S::ITER; ++it) {
    const int ya = r * S::RPR + 2 * (it * S::NG + g);
    float4 ca[8], cb[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const int kza = ka + 32 * k2, kzb = kb + 32 * k2;
      const float2 *Ca = cluster.map_shared_rank(C, kza / S::CPR);
      const float2 *Cb = cluster.map_shared_rank(C, kzb / S::CPR);
      ca[k2] = *(const float4 *)(Ca + (kza % S::CPR) * CS + ya);
      cb[k2] = *(const float4 *)(Cb + (kzb % S::CPR) * CS + ya);
    }
    float2 A[16], B[16], v[32];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      A[k2] = pack2(make_float2(ca[k2].x, ca[k2].y), make_float2(ca[k2].z, ca[k2].w));
      B[k2] = pack2(make_float2(cb[k2].x, cb[k2].y), make_float2(cb[k2].z, cb[k2].w));
    }
#pragma unroll
    for (int k2 = 8; k2 < 16; ++k2) {           // kz > 256 from the conjugate of 512 - kz
      const float4 sa = j ? cb[15 - k2] : ca[(16 - k2) & 7];
      const float4 sb = j ? ca[15 - k2] : cb[15 - k2];
      A[k2] = pack2(make_float2(sa.x, -sa.y), make_float2(sa.z, -sa.w));
      B[k2] = pack2(make_float2(sb.x, -sb.y), make_float2(sb.z, -sb.w));
    }
    if (j == 0) {                               // rank 0's packed column: (kz = 0, kz = 256) per row
      A[0] = make_float2(ca[0].x, ca[0].z);
      A[8] = make_float2(ca[0].y, ca[0].w);
    }
    inv512<S::HALF>(A, B, v, j, gm, TW, Eg);
    float *ra = plane + (long long)ya * ROWF, *rb = ra + ROWF;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      ra[16 * m + j] = v[m].x;
      rb[16 * m + j] = v[m].y;
    }
  }
  cluster_arrive();                             // no CTA leaves while others read its columns
  cluster_wait();
}

// ---------------------------------------------------------------------------
// x pass (C2C along x) through the tensor memory accelerator: mode 0 forward, 1 inverse,
// 2 forward -> * conj(D) s W^-2 -> inverse.
// The columns of a half-spectrum slot are taken in the flattened order f = ky HP + kz (x stride
// NM HP complex values; the padding column kz = 257 of every ky is transformed too, on its own).
// A tile is XC = 16 consecutive columns -- 128 contiguous bytes per row, every tile starting on
// a 128-byte boundary whatever its ky -- and all 512 rows; a slot has 132096 / 16 = 8256 tiles.  Tiles are loaded and stored by TMA in boxes of 32 rows with the
// 128-byte swizzle (16-byte chunk index XOR row % 8), so the threads issue no copy or store
// instructions of their own.  A 16-thread group (alternate lanes of a warp) transforms one
// column; the exchange of the 512-point engine runs in place in that column's own storage (slot
// (a, b) at row 16 a + (b ^ (a % 16))), which keeps every shared access of a warp at two
// wavefronts, one per half-warp.
// Persistent: one 256-thread CTA per SM.  Modes 0 and 1 keep three tile buffers.  In the x pass,
// once a tile's store is issued the load of the tile two items ahead goes into the buffer the
// previous store has left, so two loads are in flight while the CTA waits for the next tile; the
// y pass (whose tiles share DRAM rows with their neighbours) measured faster with one: its next
// tile loads while this one is transformed.  Mode 2 keeps two data
// buffers and the tile of D, walks the tile positions and, at each one, every field of the launch,
// so D is read once per launch.  Waits on the tile barriers give up after about two seconds,
// record a fault in *fault and end the kernel once the copies in flight have landed.
// ---------------------------------------------------------------------------
constexpr int XC = 16;                              // columns per tile
constexpr int XBR = 32;                             // rows per TMA box of a partial row range
constexpr int XBW = 256;                            // rows per TMA box otherwise (the largest box)
constexpr long long XNCOL = (long long)NM * HP;     // columns per slot
constexpr long long XNT = XNCOL / XC;               // tiles per slot
constexpr int YNT = (2 * HP + 2 * XC - 1) / (2 * XC);  // y pass: tiles of an x plane (16 full, 1 of kz 256, 257)
constexpr int XTILE = NM * XC * 8;                  // bytes per tile buffer
static_assert(XNCOL % XC == 0, "a slot is a whole number of tiles");

struct XtLayout {                                   // dynamic shared memory, from a 1024-byte aligned base
  static constexpr int NBUF = 3;                    // modes 0, 1: three tiles; mode 2: two tiles + the D tile
  static constexpr size_t TW_OFF = (size_t)NBUF * XTILE;
  static constexpr size_t W1_OFF = TW_OFF + sizeof(float2) * EX;
  static constexpr int NSC = 512;                   // mode 2: fields per launch (their scales s)
  static constexpr size_t SC_OFF = W1_OFF + sizeof(float) * NM;
  static constexpr size_t BAR_OFF = SC_OFF + sizeof(float) * NSC;
  static constexpr size_t BYTES = BAR_OFF + 8 * NBUF + 1024;
};

// byte offset of element (row x, column c) of a tile written with the 128-byte swizzle
__device__ __forceinline__ unsigned xt_off(int x, int c) {
  return (unsigned)(x * 128 + ((((c >> 1) ^ x) & 7) << 4) + ((c & 1) << 3));
}

struct XtCol {                                      // one column of a swizzled tile
  unsigned char *tile;
  int c;
  __device__ __forceinline__ float2 &at(int x) const { return *(float2 *)(tile + xt_off(x, c)); }
  __device__ __forceinline__ float2 &operator()(int a, int b) const { return at(16 * a + (b ^ (a & 15))); }
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase of the given parity to complete; false after about two seconds
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 2000000000ull) return false;
  return true;
}
__device__ __forceinline__ void tma_load(unsigned char *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap *map, int c0, int c1, int c2, const unsigned char *src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
               ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The tiles of a launch of modes 0 and 1: nslab slabs of ntile tiles, slab q at the third
// tensor-map coordinate (q / np) sstride + s0 + q % np.  x pass: one slab per slot (ntile = XNT,
// np = sstride = 1, s0 = 0); y pass: the x planes [s0, s0 + np) of every slot (sstride = NM,
// ntile = YNT tiles of 16 kz columns, the rows being ky).
struct XtUnits {
  long long nslab;
  int ntile, np, sstride, s0;
  int ahead;       // modes 0, 1: tiles loading ahead of the one transformed (2: x pass, 1: y pass)
};

template <int MODE>
__global__ void __launch_bounds__(256, 1)
    fft512_xt(const __grid_constant__ CUtensorMap tm, const __grid_constant__ CUtensorMap tmw,
              const __grid_constant__ CUtensorMap tmd, int nslots,
              XtUnits un, const float2 *__restrict__ gtw, const double *__restrict__ scale,
              const float *__restrict__ invw, int xlo, int xhi, unsigned *__restrict__ fault) {
  using L = XtLayout;
  extern __shared__ __align__(16) unsigned char smraw[];
  // 1024-byte aligned base (the 128-byte swizzle repeats every 8 rows); pointer arithmetic on the
  // shared array keeps every access below a shared-memory instruction
  unsigned char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  float2 *TW = (float2 *)(sm + L::TW_OFF);
  float *W1 = (float *)(sm + L::W1_OFF);
  float *SC = (float *)(sm + L::SC_OFF);
  unsigned long long *bar = (unsigned long long *)(sm + L::BAR_OFF);
  // the two groups of a warp take alternate lanes: a column of a tile uses one 8-byte half of each
  // 16-byte chunk, so each half-warp (which the 8-byte accesses are served by) then covers both
  // halves of 8 chunks -- 16 different bank pairs, one wavefront -- where a whole group in one
  // half-warp would meet each bank pair twice
  const int tid = threadIdx.x, lane = tid & 31, g = 2 * (tid >> 5) + (lane & 1), j = lane >> 1;
  const unsigned gm = 0x55555555u << (lane & 1);
  const int ka = j, kb = col_b(j);
  const int lo = MODE == 1 ? 0 : xlo, hi = MODE == 1 ? NM : xhi;   // rows read from HBM
  const long long nunits = MODE == 2 ? XNT : un.nslab * un.ntile;
  const int nf = MODE == 2 ? nslots : 1;
  constexpr int NDB = MODE == 2 ? 2 : 3;            // data buffers

  if (tid == 0) {
    for (int b = 0; b < L::NBUF; ++b) mbar_init(bar + b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < EX; i += blockDim.x) TW[i] = gtw[i];
  if (MODE == 2 && invw)
    for (int i = tid; i < NM; i += blockDim.x) W1[i] = invw[i];
  if (MODE == 2)
    for (int i = tid; i < nf; i += blockDim.x) SC[i] = (float)scale[i];
  __syncthreads();
  const TabTw ttw{TW, j, kb};   // twiddles read from the shared table (no registers held for them)

  // item i = (unit u, field f): modes 0, 1 take the tiles of every slot (f = 0), mode 2 the
  // positions with every field; data buffer i % NDB, whose barrier completes once per use
  // tensor-map coordinates of item (u, f): c0 (floats along a row of tiles) and c2 (slot or plane)
  auto coords = [&](long long u, int f, int &c0, int &c2) {
    if (MODE == 2) {
      c0 = (int)(u * (2 * XC));
      c2 = f;
    } else {
      const long long q = u / un.ntile;
      c0 = (int)(u % un.ntile) * (2 * XC);
      c2 = (int)(q / un.np) * un.sstride + un.s0 + (int)(q % un.np);
    }
  };
  auto issue_data = [&](long long u, int f, int b) {
    int c0, c2;
    coords(u, f, c0, c2);
    mbar_expect_tx(bar + b, (unsigned)(hi - lo) * 128u);
    for (int x0 = lo; x0 < hi;) {                   // boxes of XBW rows where they fit, else XBR
      const bool wide = MODE != 2 && (x0 % XBW) == 0 && x0 + XBW <= hi;
      tma_load(sm + (size_t)b * XTILE + (size_t)x0 * 128, wide ? &tmw : &tm, c0, x0, c2, bar + b);
      x0 += wide ? XBW : XBR;
    }
  };
  auto issue_d = [&](long long u) {
    mbar_expect_tx(bar + 2, (unsigned)NM * 128u);
    for (int x0 = 0; x0 < NM; x0 += XBR)
      tma_load(sm + (size_t)2 * XTILE + (size_t)x0 * 128, &tmd, (int)(u * (2 * XC)), x0, 0, bar + 2);
  };
  // pending loads (bit b: buffer b), and the parity each one completes with, for a clean exit
  unsigned pend = 0, ppar = 0;
  long long u = blockIdx.x;
  if (tid == 0 && u < nunits) {
    issue_data(u, 0, 0);
    pend |= 1u;
    if (MODE == 2) {
      issue_d(u);
      pend |= 4u;
    } else if (un.ahead == 2 && u + gridDim.x < nunits) {   // two tiles ahead from the start
      issue_data(u + gridDim.x, 0, 1);
      pend |= 2u;
    }
  }
  bool ok = true;
  long long i = 0;
  for (long long k = 0; u < nunits && ok; u += gridDim.x, ++k) {
    for (int f = 0; f < nf && ok; ++f, ++i) {
      const int b = (int)(i % NDB);
      const unsigned par = (unsigned)((i / NDB) & 1);
      bool w = mbar_wait(bar + b, par);
      if (MODE == 2 && f == 0) w = w && mbar_wait(bar + 2, (unsigned)(k & 1));
      ok = __syncthreads_and(w);
      if (!ok) break;
      if (tid == 0) {
        pend &= ~(1u << b);
        if (MODE == 2 && f == 0) pend &= ~4u;
      }
      unsigned char *tile = sm + (size_t)b * XTILE;
      if ((MODE == 2 || un.ahead == 1) && tid == 0) {   // prefetch the next item
        long long un = u;
        int fn = f + 1;
        if (fn >= nf) {
          un = u + gridDim.x;
          fn = 0;
        }
        if (un < nunits) {
          const int bn = (int)((i + 1) % NDB);
          if (MODE == 2)
            bulk_wait_read<0>();                     // the store of item i - 1 (buffer bn) has read its tile
          else
            bulk_wait_read<1>();                     // the store of item i - 2 (buffer bn) has read its tile
          issue_data(un, fn, bn);
          pend |= 1u << bn;
          ppar = (ppar & ~(1u << bn)) | ((unsigned)(((i + 1) / NDB) & 1) << bn);
        }
      }
      const long long tl = u;                        // mode 2: the tile position
      const XtCol col{tile, g};
      float2 v[32], As[16], Bs[16];
      const float s = MODE == 2 ? SC[f] : 1.f;
      if (MODE == 1) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          As[k2] = col.at(ka + 32 * k2);
          Bs[k2] = col.at(kb + 32 * k2);
        }
      } else {
        // rows outside [lo, hi) hold no painted value and were not loaded: lo and hi are multiples
        // of 32, so row 16 m + j lies in the range exactly when m does in [lo / 16, hi / 16)
        const int mlo = lo >> 4, mhi = hi >> 4;
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = (m >= mlo && m < mhi) ? col.at(16 * m + j) : make_float2(0.f, 0.f);
        fwd512x(v, As, Bs, j, gm, ttw, col);
      }
      if (MODE == 2) {
        const XtCol dcol{sm + (size_t)2 * XTILE, g};
        if (f == 0) {
          // D <- conj(D) W^-2 in place, once per position: every thread rewrites exactly the
          // entries kx = ka + 32 k2, kb + 32 k2 of its column that it reads below
          const long long fc = tl * XC + g;
          const int ky = (int)(fc / HP), kz = (int)(fc % HP);
          const float cyz = invw ? W1[ky] * W1[kz] : 1.f;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int kxa = ka + 32 * k2, kxb = kb + 32 * k2;
            float wa = 1.f, wb = 1.f;
            if (invw) {
              wa = W1[kxa] * cyz;
              wb = W1[kxb] * cyz;
            }
            dcol.at(kxa) = cscale(cconj(dcol.at(kxa)), wa * wa);
            dcol.at(kxb) = cscale(cconj(dcol.at(kxb)), wb * wb);
          }
        }
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          As[k2] = cscale(cmul(As[k2], dcol.at(ka + 32 * k2)), s);
          Bs[k2] = cscale(cmul(Bs[k2], dcol.at(kb + 32 * k2)), s);
        }
      }
      if (MODE == 0) {
        __syncwarp(gm);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          col.at(ka + 32 * k2) = As[k2];
          col.at(kb + 32 * k2) = Bs[k2];
        }
      } else {
        inv512x(As, Bs, v, j, gm, ttw, col);
        __syncwarp(gm);
#pragma unroll
        for (int m = 0; m < 32; ++m) col.at(16 * m + j) = v[m];
      }
      fence_async_smem();                            // these writes (and D's rewrite) before async-proxy use
      __syncthreads();
      if (tid == 0) {
        int c0, c2;
        coords(u, f, c0, c2);
        // wide boxes in modes 0 and 1; the convolution pass measured faster with narrow ones
        if (MODE == 2)
          for (int x0 = 0; x0 < NM; x0 += XBR) tma_store(&tm, c0, x0, c2, tile + (size_t)x0 * 128);
        else
          for (int x0 = 0; x0 < NM; x0 += XBW) tma_store(&tmw, c0, x0, c2, tile + (size_t)x0 * 128);
        bulk_commit();
        if (MODE != 2 && un.ahead == 2 && u + 2 * gridDim.x < nunits) {   // the tile two items ahead
          const int b2 = (int)((i + 2) % NDB);
          bulk_wait_read<1>();                       // the store of item i - 1 (buffer b2) has read its tile
          issue_data(u + 2 * gridDim.x, 0, b2);
          pend |= 1u << b2;
          ppar = (ppar & ~(1u << b2)) | ((unsigned)(((i + 2) / NDB) & 1) << b2);
        }
        if (MODE == 2 && f == nf - 1 && u + gridDim.x < nunits) {   // D of the next position
          issue_d(u + gridDim.x);
          pend |= 4u;
          ppar = (ppar & ~4u) | ((unsigned)((k + 1) & 1) << 2);
        }
      }
    }
  }
  if (tid == 0) {
    if (!ok) {
      *(volatile unsigned *)fault = 1u;
      for (int b = 0; b < L::NBUF; ++b)              // let the loads in flight land before leaving
        if (pend & (1u << b)) mbar_wait(bar + b, (ppar >> b) & 1u);
    }
    bulk_wait_all();
  }
}

// ---------------------------------------------------------------------------
// z pass (R2C / C2R along z of whole rows).  A unit is a block of ZR = 32 consecutive rows of
// one x plane: 66048 contiguous bytes (the 2064-byte rows start on 16-byte boundaries), moved by
// one bulk copy each way.  A 16-thread group (16 consecutive lanes) transforms the row pair
// (2 g, 2 g + 1) of the block as the complex sequence a + i b; the engine's exchange runs in
// place in the pair's own 4128 bytes (slot (a, b) at float2 16 a + (b ^ (a % 16)), one
// wavefront per half-warp with this row pitch).  Forward: the two half spectra are separated in
// registers (X[k] and X[512 - k] sit in the same thread) and written over the rows, kz = 0..256;
// inverse: the rows' half spectra are joined into one sequence, completed by Hermitian symmetry
// in registers, and transformed back.  Persistent, one 256-thread CTA per SM, three block
// buffers (load of the next block, transform of this one, store of the previous one in flight);
// waits give up after about two seconds like the x pass's.
// ---------------------------------------------------------------------------
constexpr int ZR = 32;                                   // rows per unit
constexpr unsigned ZBLK = (unsigned)(ZR * ROWF * 4);     // 66048 bytes per block

struct ZtLayout {
  static constexpr int NBUF = 3;
  static constexpr size_t TW_OFF = (size_t)NBUF * ZBLK;
  static constexpr size_t BAR_OFF = TW_OFF + sizeof(float2) * EX;
  static constexpr size_t BYTES = BAR_OFF + 8 * NBUF + 128;
};

struct RowEx {                                           // exchange slots of one row pair, in place
  float2 *p;
  __device__ __forceinline__ float2 &operator()(int a, int b) const { return p[16 * a + (b ^ (a & 15))]; }
};

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}

// units: the row blocks [ylo / ZR, ylo / ZR + nyb) of the x planes [xlo, xlo + np) of nslots slots
template <int INV>
__global__ void __launch_bounds__(256, 1)
    fft512_zt(float *__restrict__ data, long long slot_reals, int nslots, int xlo, int np, int ylo, int nyb,
              const float2 *__restrict__ gtw, unsigned *__restrict__ fault) {
  using L = ZtLayout;
  extern __shared__ __align__(16) unsigned char smz[];
  unsigned char *sm = smz + ((128u - (smem_u32(smz) & 127u)) & 127u);
  float2 *TW = (float2 *)(sm + L::TW_OFF);
  unsigned long long *bar = (unsigned long long *)(sm + L::BAR_OFF);
  const int tid = threadIdx.x, g = tid >> 4, j = tid & 15;
  const unsigned gm = 0xFFFFu << (tid & 16);
  const int ka = j, kb = col_b(j);
  const long long nunits = (long long)nslots * np * nyb;

  if (tid == 0) {
    for (int b = 0; b < L::NBUF; ++b) mbar_init(bar + b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < EX; i += blockDim.x) TW[i] = gtw[i];
  __syncthreads();
  const TabTw tw{TW, j, kb};    // twiddles read from the shared table

  auto block = [&](long long u) -> float * {
    const long long q = u / nyb;
    const int s = (int)(q / np), x = xlo + (int)(q % np), y0 = ylo + (int)(u % nyb) * ZR;
    return data + (long long)s * slot_reals + ((long long)x * NM + y0) * ROWF;
  };
  auto issue = [&](long long u, int b) {
    mbar_expect_tx(bar + b, ZBLK);
    bulk_load(sm + (size_t)b * ZBLK, block(u), ZBLK, bar + b);
  };
  unsigned pend = 0, ppar = 0;
  long long u = blockIdx.x;
  if (tid == 0 && u < nunits) {
    issue(u, 0);
    pend |= 1u;
  }
  bool ok = true;
  for (long long k = 0; u < nunits; u += gridDim.x, ++k) {
    const int b = (int)(k % L::NBUF);
    const unsigned par = (unsigned)((k / L::NBUF) & 1);
    ok = __syncthreads_and(mbar_wait(bar + b, par));
    if (!ok) break;
    if (tid == 0) {
      pend &= ~(1u << b);
      const long long un = u + gridDim.x;
      if (un < nunits) {                             // prefetch the next block
        const int bn = (int)((k + 1) % L::NBUF);
        bulk_wait_read<1>();                         // the store of block k - 2 (buffer bn) has read it
        issue(un, bn);
        pend |= 1u << bn;
        ppar = (ppar & ~(1u << bn)) | ((unsigned)(((k + 1) / L::NBUF) & 1) << bn);
      }
    }
    float *blk = (float *)(sm + (size_t)b * ZBLK);
    float *ra = blk + (size_t)(2 * g) * ROWF, *rb = ra + ROWF;
    float2 *pa = (float2 *)ra, *pb = (float2 *)rb;
    const RowEx ex{pa};
    float2 v[32], A[16], B[16];
    if (!INV) {
#pragma unroll
      for (int m = 0; m < 32; ++m) v[m] = make_float2(ra[16 * m + j], rb[16 * m + j]);
      fwd512x(v, A, B, j, gm, tw, ex);
      __syncwarp(gm);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {               // kz = ka + 32 k2, kb + 32 k2: 0..255
        const float4 va = unpack2(A[k2], j ? cconj(B[15 - k2]) : cconj(A[(16 - k2) & 15]));
        const float4 vb = unpack2(B[k2], j ? cconj(A[15 - k2]) : cconj(B[15 - k2]));
        pa[ka + 32 * k2] = make_float2(va.x, va.y);
        pb[ka + 32 * k2] = make_float2(va.z, va.w);
        pa[kb + 32 * k2] = make_float2(vb.x, vb.y);
        pb[kb + 32 * k2] = make_float2(vb.z, vb.w);
      }
      if (j == 0) {                                  // kz = 256
        const float4 vn = unpack2(A[8], cconj(A[8]));
        pa[256] = make_float2(vn.x, vn.y);
        pb[256] = make_float2(vn.z, vn.w);
      }
    } else {
      float4 ca[8], cb[8];                           // (row a, row b) at kz = ka + 32 k2, kb + 32 k2
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        const float2 a0 = pa[ka + 32 * k2], b0 = pb[ka + 32 * k2], a1 = pa[kb + 32 * k2], b1 = pb[kb + 32 * k2];
        ca[k2] = make_float4(a0.x, a0.y, b0.x, b0.y);
        cb[k2] = make_float4(a1.x, a1.y, b1.x, b1.y);
      }
      const float2 a256 = pa[256], b256 = pb[256];
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        A[k2] = pack2(make_float2(ca[k2].x, ca[k2].y), make_float2(ca[k2].z, ca[k2].w));
        B[k2] = pack2(make_float2(cb[k2].x, cb[k2].y), make_float2(cb[k2].z, cb[k2].w));
      }
#pragma unroll
      for (int k2 = 8; k2 < 16; ++k2) {              // kz > 256 from the conjugate at 512 - kz
        const float4 sa = j ? cb[15 - k2] : ca[(16 - k2) & 7];
        const float4 sb = j ? ca[15 - k2] : cb[15 - k2];
        A[k2] = pack2(make_float2(sa.x, -sa.y), make_float2(sa.z, -sa.w));
        B[k2] = pack2(make_float2(sb.x, -sb.y), make_float2(sb.z, -sb.w));
      }
      if (j == 0) A[8] = pack2(a256, b256);          // kz = 256 (its own conjugate partner)
      __syncwarp(gm);                                // every spectrum read before the exchange
      inv512x(A, B, v, j, gm, tw, ex);
      __syncwarp(gm);
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        ra[16 * m + j] = v[m].x;
        rb[16 * m + j] = v[m].y;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_store(block(u), blk, ZBLK);
      bulk_commit();
    }
  }
  if (tid == 0) {
    if (!ok) {
      *(volatile unsigned *)fault = 1u;
      for (int b = 0; b < L::NBUF; ++b)
        if (pend & (1u << b)) mbar_wait(bar + b, (ppar >> b) & 1u);
    }
    bulk_wait_all();
  }
}

float2 *g_twiddles[64] = {nullptr};
std::mutex g_tw_mu;

const float2 *twiddles(int dev) {
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (!g_twiddles[dev]) {
    float2 host[EX];
    for (int k1 = 0; k1 < 32; ++k1)
      for (int j = 0; j < ES; ++j) {
        const double a = -2.0 * M_PI * (double)(k1 * j) / 512.0;
        host[k1 * ES + j] = j < 16 ? make_float2((float)std::cos(a), (float)std::sin(a)) : make_float2(0.f, 0.f);
      }
    float2 *d = nullptr;
    if (cudaMalloc(&d, sizeof host) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, host, sizeof host, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(d);
      return nullptr;
    }
    g_twiddles[dev] = d;
  }
  return g_twiddles[dev];
}

template <int CL>
cudaError_t plane_attrs() {
  cudaError_t e;
  const int smem = (int)PlaneShape<CL>::SMEM;
  if ((e = cudaFuncSetAttribute(fft512_plane_fwd<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(fft512_plane_inv<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  if (CL > 8) {
    if ((e = cudaFuncSetAttribute(fft512_plane_fwd<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_plane_inv<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

template <int CL>
cudaError_t launch_plane(bool inverse, float *b, long long slot_reals, int n, const float2 *tw, cudaStream_t st) {
  using S = PlaneShape<CL>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, NM, n);
  cfg.blockDim = dim3(S::NT, 1, 1);
  cfg.dynamicSmemBytes = S::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return inverse ? cudaLaunchKernelEx(&cfg, fft512_plane_inv<CL>, b, slot_reals, tw)
                 : cudaLaunchKernelEx(&cfg, fft512_plane_fwd<CL>, b, slot_reals, tw);
}

cudaError_t plane(int cluster, bool inverse, float *b, long long slot_reals, int n, const float2 *tw,
                  cudaStream_t st) {
  return cluster == 16 ? launch_plane<16>(inverse, b, slot_reals, n, tw, st)
                       : launch_plane<8>(inverse, b, slot_reals, n, tw, st);
}

int sm_count(int dev) {
  static int n[64] = {0};
  if (!n[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    n[dev] = v;
  }
  return n[dev];
}

// per device: a word of mapped host memory that an x pass sets when a tile wait gives up
// (device view g_xfault, host view g_xfault_host: the host reads it without a CUDA call)
unsigned *g_xfault[64] = {nullptr};
volatile unsigned *g_xfault_host[64] = {nullptr};

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// TMA map of n half-spectrum slots from base b: dims (2 NM HP floats of an x-plane, NM planes, n slots),
// boxes of 32 floats (16 complex columns, 128 bytes) x `rows` planes x 1 slot, 128-byte swizzle
cudaError_t slot_map(CUtensorMap *m, float *b, long long slot_reals, int n, int rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * XNCOL), (cuuint64_t)NM, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * XNCOL * sizeof(float)), (cuuint64_t)(slot_reals * sizeof(float))};
  const cuuint32_t box[3] = {2 * XC, (cuuint32_t)rows, 1}, estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, b, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t xpass(float *b, long long slot_reals, int n, const float2 *tw, const float *D, const double *scale,
                  const float *invw, cudaStream_t st, int xlo = 0, int xhi = NM) {
  if (xlo < 0 || xhi > NM || xlo >= xhi || xlo % XBR || xhi % XBR) return cudaErrorInvalidValue;
  if (((unsigned long long)b & 15ull) || (MODE == 2 && ((unsigned long long)D & 15ull)) ||
      (slot_reals * sizeof(float)) % 16)
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaGetDevice(&dev);
  CUtensorMap tm, tmw, tmd;
  cudaError_t e = slot_map(&tm, b, slot_reals, n, XBR);
  if (e == cudaSuccess) e = slot_map(&tmw, b, slot_reals, n, XBW);
  if (e == cudaSuccess) e = slot_map(&tmd, MODE == 2 ? (float *)D : b, slot_reals, 1, XBR);
  if (e != cudaSuccess) return e;
  if (MODE == 2 && n > XtLayout::NSC) return cudaErrorInvalidValue;
  const long long units = MODE == 2 ? XNT : XNT * n;
  const long long grid = std::min<long long>(units, (long long)sm_count(dev));
  const XtUnits un{(long long)n, (int)XNT, 1, 1, 0, 2};
  fft512_xt<MODE><<<(unsigned)grid, 256, XtLayout::BYTES, st>>>(tm, tmw, tmd, n, un, tw, scale, invw, xlo, xhi,
                                                                g_xfault[dev]);
  return cudaGetLastError();
}

// TMA map of the x planes of n slots from base b for the y pass: dims (2 HP floats of a row, NM
// rows ky, NM n planes), the row stride 2064 bytes (a multiple of 16, which the padded layout
// exists for) and the plane stride NM rows; boxes of 32 floats x `rows` rows x 1 plane, 128-byte
// swizzle.  The last tile of a row (kz 256 and the padding) lies partly outside dimension 0:
// its loads read zeros there and its stores skip it.
cudaError_t plane_map(CUtensorMap *m, float *b, int n, int rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)ROWF, (cuuint64_t)NM, (cuuint64_t)NM * (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)(ROWF * sizeof(float)), (cuuint64_t)(NM * ROWF * sizeof(float))};
  const cuuint32_t box[3] = {2 * XC, (cuuint32_t)rows, 1}, estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, b, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// y pass (C2C along y) of the x planes [xlo, xhi) of n slots; mode 0 (forward) reads the rows
// y in [ylo, yhi) only, mode 1 (inverse) every row
template <int MODE>
cudaError_t ypass(float *b, long long slot_reals, int n, const float2 *tw, cudaStream_t st, int xlo, int xhi, int ylo,
                  int yhi) {
  static_assert(MODE == 0 || MODE == 1, "forward or inverse");
  if (xlo < 0 || xhi > NM || xlo >= xhi || ylo < 0 || yhi > NM || ylo >= yhi || ylo % XBR || yhi % XBR)
    return cudaErrorInvalidValue;
  if (((unsigned long long)b & 15ull) || slot_reals != (long long)NM * NM * ROWF) return cudaErrorInvalidValue;
  int dev = 0;
  cudaGetDevice(&dev);
  CUtensorMap tm, tmw;
  cudaError_t e = plane_map(&tm, b, n, XBR);
  if (e == cudaSuccess) e = plane_map(&tmw, b, n, XBW);
  if (e != cudaSuccess) return e;
  const XtUnits un{(long long)n * (xhi - xlo), YNT, xhi - xlo, NM, xlo, 1};
  const long long grid = std::min<long long>(un.nslab * YNT, (long long)sm_count(dev));
  fft512_xt<MODE><<<(unsigned)grid, 256, XtLayout::BYTES, st>>>(tm, tmw, tmw, n, un, tw, nullptr, nullptr, ylo, yhi,
                                                                g_xfault[dev]);
  return cudaGetLastError();
}

// z pass of the rows y in [ylo, yhi) of the x planes [xlo, xhi) of n slots
template <int INV>
cudaError_t zpass(float *b, long long slot_reals, int n, const float2 *tw, cudaStream_t st, int xlo, int xhi, int ylo,
                  int yhi) {
  if (xlo < 0 || xhi > NM || xlo >= xhi || ylo < 0 || yhi > NM || ylo >= yhi || ylo % ZR || yhi % ZR)
    return cudaErrorInvalidValue;
  if (((unsigned long long)b & 15ull) || slot_reals != (long long)NM * NM * ROWF) return cudaErrorInvalidValue;
  int dev = 0;
  cudaGetDevice(&dev);
  const int np = xhi - xlo, nyb = (yhi - ylo) / ZR;
  const long long units = (long long)n * np * nyb;
  const long long grid = std::min<long long>(units, (long long)sm_count(dev));
  fft512_zt<INV><<<(unsigned)grid, 256, ZtLayout::BYTES, st>>>(b, slot_reals, n, xlo, np, ylo, nyb, tw,
                                                               g_xfault[dev]);
  return cudaGetLastError();
}

}  // namespace

bool native_fft_supported(int n_mesh, int precision) { return n_mesh == NM && precision == 32; }

cudaError_t native_fft_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!twiddles(dev)) return cudaErrorMemoryAllocation;
  static bool attrs[64] = {false};
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (!attrs[dev]) {
    if ((e = plane_attrs<8>()) != cudaSuccess) return e;
    if ((e = plane_attrs<16>()) != cudaSuccess) return e;
    const int xs = (int)XtLayout::BYTES;
    if ((e = cudaFuncSetAttribute(fft512_xt<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, xs)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_xt<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, xs)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_xt<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, xs)) != cudaSuccess)
      return e;
    const int zs = (int)ZtLayout::BYTES;
    if ((e = cudaFuncSetAttribute(fft512_zt<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, zs)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fft512_zt<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, zs)) != cudaSuccess)
      return e;
    if (!tensor_map_encoder()) return cudaErrorNotSupported;
    unsigned *hf = nullptr;
    if ((e = cudaHostAlloc((void **)&hf, sizeof(unsigned), cudaHostAllocMapped)) != cudaSuccess) return e;
    *hf = 0;
    if ((e = cudaHostGetDevicePointer((void **)&g_xfault[dev], hf, 0)) != cudaSuccess) return e;
    g_xfault_host[dev] = hf;
    attrs[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t native_fft_forward(float *slots, long long slot_reals, int first, int count, int cluster,
                               cudaStream_t st) {
  if (cluster != 8 && cluster != 16) return cudaErrorInvalidValue;
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  cudaError_t e = cudaSuccess;
  for (int done = 0; done < count && e == cudaSuccess; done += 65535) {
    const int n = count - done < 65535 ? count - done : 65535;
    float *b = base + (long long)done * slot_reals;
    if ((e = plane(cluster, false, b, slot_reals, n, tw, st)) == cudaSuccess)
      e = xpass<0>(b, slot_reals, n, tw, nullptr, nullptr, nullptr, st);
  }
  return e;
}

cudaError_t native_fft_inverse(float *slots, long long slot_reals, int first, int count, int cluster,
                               cudaStream_t st) {
  if (cluster != 8 && cluster != 16) return cudaErrorInvalidValue;
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  cudaError_t e = cudaSuccess;
  for (int done = 0; done < count && e == cudaSuccess; done += 65535) {
    const int n = count - done < 65535 ? count - done : 65535;
    float *b = base + (long long)done * slot_reals;
    if ((e = xpass<1>(b, slot_reals, n, tw, nullptr, nullptr, nullptr, st)) == cudaSuccess)
      e = plane(cluster, true, b, slot_reals, n, tw, st);
  }
  return e;
}

cudaError_t native_fft_xpass(int mode, float *slots, long long slot_reals, int first, int count, const float *D,
                             const double *scale, const float *invw, cudaStream_t st, int xlo, int xhi) {
  if (mode < 0 || mode > 2 || (mode == 2 && (!D || !scale))) return cudaErrorInvalidValue;
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  cudaError_t e = cudaSuccess;
  const int step = mode == 2 ? XtLayout::NSC : 65535;
  for (int done = 0; done < count && e == cudaSuccess; done += step) {
    const int n = count - done < step ? count - done : step;
    float *b = base + (long long)done * slot_reals;
    e = mode == 0   ? xpass<0>(b, slot_reals, n, tw, nullptr, nullptr, nullptr, st, xlo, xhi)
        : mode == 1 ? xpass<1>(b, slot_reals, n, tw, nullptr, nullptr, nullptr, st)
                    : xpass<2>(b, slot_reals, n, tw, D, scale + done, invw, st, xlo, xhi);
  }
  return e;
}

cudaError_t native_fft_zpass(int inverse, float *slots, long long slot_reals, int first, int count, cudaStream_t st,
                             int xlo, int xhi, int ylo, int yhi) {
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  return inverse ? zpass<1>(slots + (long long)first * slot_reals, slot_reals, count, tw, st, xlo, xhi, ylo, yhi)
                 : zpass<0>(slots + (long long)first * slot_reals, slot_reals, count, tw, st, xlo, xhi, ylo, yhi);
}

cudaError_t native_fft_ypass(int inverse, float *slots, long long slot_reals, int first, int count, cudaStream_t st,
                             int xlo, int xhi, int ylo, int yhi) {
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  cudaError_t e = cudaSuccess;
  const int step = 65535 / NM;                       // planes of a launch fit a 16-bit count
  for (int done = 0; done < count && e == cudaSuccess; done += step) {
    const int n = count - done < step ? count - done : step;
    float *b = base + (long long)done * slot_reals;
    e = inverse ? ypass<1>(b, slot_reals, n, tw, st, xlo, xhi, ylo, yhi)
                : ypass<0>(b, slot_reals, n, tw, st, xlo, xhi, ylo, yhi);
  }
  return e;
}

bool native_fft_fault(int dev) { return dev >= 0 && dev < 64 && g_xfault_host[dev] && *g_xfault_host[dev] != 0u; }

cudaError_t native_fft_convolve(float *slots, long long slot_reals, int first, int count, const float *D,
                                const double *scale, const float *invw, int cluster, cudaStream_t st) {
  if (cluster != 8 && cluster != 16) return cudaErrorInvalidValue;
  if (count <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const float2 *tw = twiddles(dev);
  float *base = slots + (long long)first * slot_reals;
  cudaError_t e = cudaSuccess;
  for (int done = 0; done < count && e == cudaSuccess; done += XtLayout::NSC) {
    const int n = count - done < XtLayout::NSC ? count - done : XtLayout::NSC;
    float *b = base + (long long)done * slot_reals;
    if ((e = plane(cluster, false, b, slot_reals, n, tw, st)) != cudaSuccess) break;
    if ((e = xpass<2>(b, slot_reals, n, tw, D, scale + done, invw, st)) != cudaSuccess) break;
    e = plane(cluster, true, b, slot_reals, n, tw, st);
  }
  return e;
}

}  // namespace bym
