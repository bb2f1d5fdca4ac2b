// Ahead-of-time kernels of the mesh front end and the spectral products.
//
//   bym_norm_reduce   FP64 sums of w_g, w_r, nbar_r w_r^2 and a count of objects
//                     outside the box (Sec. 2.1: alpha_r and the FKP normalisation);
//   bym_paint         CIC / TSC mass assignment of signed weights w and -alpha_r w
//                     into the padded real mesh (periodic, FP64 cell geometry);
//   bym_spec_mul      F(k) <- F(k) conj(delta(k)) s_f W(k)^-2 for a run of field
//                     spectra (the convolution step of eq. g-JM-form / eq. 2pcf-yama);
//   bym_spec_mul_cross  the same step for two tracers: F^A(k) <- [F^A(k) conj(delta_B(k))
//                     + F^B(k) conj(delta_A(k))] s_f W(k)^-2 / 2 (both anchorings of the
//                     midpoint series, and the two endpoint lines of sight of Yamamoto);
//   bym_interlace     F(k) <- (F(k) + P(k) G(k)) / 2 with G the transform on the mesh
//                     shifted by half a cell (interlaced mass assignment).
#include "kernels.cuh"

namespace bym {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ void atomic_add(T *p, T v) {
  atomicAdd(p, v);
}

}  // namespace

// stats[0] += sum w (galaxies, which = 0) or stats[1] += sum w (randoms, which = 1);
// randoms also add stats[2] += sum nbar w^2 (nbar may be null: 0); stats[3] counts
// objects whose position is not finite or lies outside [lo, lo + N h);
// stats[4 + which] += sum w^2 (the shot-noise level of Sec. 2.1).
__global__ void __launch_bounds__(256) bym_norm_reduce(const float4 *__restrict__ p, const float *__restrict__ nbar,
                                                       long long n, int which, double lo0, double lo1, double lo2,
                                                       double inv_h, int N, double *__restrict__ stats) {
  double sw = 0.0, snw2 = 0.0, bad = 0.0, sw2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 q = p[i];
    const double ux = ((double)q.x - lo0) * inv_h, uy = ((double)q.y - lo1) * inv_h, uz = ((double)q.z - lo2) * inv_h;
    const bool ok = (ux >= 0.0) && (ux < N) && (uy >= 0.0) && (uy < N) && (uz >= 0.0) && (uz < N) &&
                    isfinite((double)q.w);
    if (!ok) bad += 1.0;
    sw += (double)q.w;
    sw2 += (double)q.w * (double)q.w;
    if (which == 1 && nbar) snw2 += (double)nbar[i] * (double)q.w * (double)q.w;
  }
  __shared__ double red[4][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  sw = warp_sum(sw);
  snw2 = warp_sum(snw2);
  bad = warp_sum(bad);
  sw2 = warp_sum(sw2);
  if (lane == 0) {
    red[0][wid] = sw;
    red[1][wid] = snw2;
    red[2][wid] = bad;
    red[3][wid] = sw2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0, d = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
      d += red[3][w];
    }
    atomicAdd(stats + 4 + which, d);
    atomicAdd(stats + which, a);
    if (which == 1) atomicAdd(stats + 2, b);
    if (c != 0.0) atomicAdd(stats + 3, c);
  }
}

// One thread per object.  Galaxies carry +w, randoms -alpha_r w with
// alpha_r = stats[0] / stats[1] read on the device.  Objects outside the box
// are skipped (the call reports them as an error).  shift (in cells, 0 or 1/2):
// paint onto the nodes box_lo + (i + shift) h, periodically (interlacing).
template <typename T>
__global__ void __launch_bounds__(256) bym_paint(const float4 *__restrict__ p, long long n, int is_ran,
                                                 const double *__restrict__ stats, T *__restrict__ delta, int N,
                                                 double lo0, double lo1, double lo2, double inv_h, int assign,
                                                 double shift) {
  const double scale = is_ran ? -(stats[0] / stats[1]) : 1.0;
  const long long row = (long long)(N + 2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 q = p[i];
    const double u[3] = {((double)q.x - lo0) * inv_h, ((double)q.y - lo1) * inv_h, ((double)q.z - lo2) * inv_h};
    if (!(u[0] >= 0.0 && u[0] < N && u[1] >= 0.0 && u[1] < N && u[2] >= 0.0 && u[2] < N)) continue;
    const double w = scale * (double)q.w;
    if (assign == 2) {
      int b[3];
      double f[3];
      for (int a = 0; a < 3; ++a) {
        const double us = u[a] - shift;
        const double fl = floor(us);
        b[a] = (int)fl;
        f[a] = us - fl;
      }
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        const int ix = (b[0] + ox + N) % N;
        const double wx = ox ? f[0] : 1.0 - f[0];
#pragma unroll
        for (int oy = 0; oy < 2; ++oy) {
          const int iy = (b[1] + oy + N) % N;
          const double wy = oy ? f[1] : 1.0 - f[1];
#pragma unroll
          for (int oz = 0; oz < 2; ++oz) {
            const int iz = (b[2] + oz + N) % N;
            const double wz = oz ? f[2] : 1.0 - f[2];
            atomic_add(delta + ((long long)ix * N + iy) * row + iz, (T)(w * wx * wy * wz));
          }
        }
      }
    } else {
      int b[3];
      double wt[3][3];
      for (int a = 0; a < 3; ++a) {
        const double us = u[a] - shift;
        const double fl = floor(us + 0.5);
        b[a] = (int)fl;
        const double d = us - fl;
        wt[a][0] = 0.5 * (0.5 - d) * (0.5 - d);
        wt[a][1] = 0.75 - d * d;
        wt[a][2] = 0.5 * (0.5 + d) * (0.5 + d);
      }
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        const int ix = (b[0] + ox + N) % N;
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
          const int iy = (b[1] + oy + N) % N;
#pragma unroll
          for (int oz = -1; oz <= 1; ++oz) {
            const int iz = (b[2] + oz + N) % N;
            atomic_add(delta + ((long long)ix * N + iy) * row + iz,
                       (T)(w * wt[0][ox + 1] * wt[1][oy + 1] * wt[2][oz + 1]));
          }
        }
      }
    }
  }
}

// F_f(k) <- F_f(k) conj(D(k)) scale[f] c(k), f = 0..nf-1 (slots of cslot complex
// values each), c = prod_axis invw^2 (compensation, null: 1).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) bym_spec_mul(T2 *__restrict__ F, long long cslot, int nf,
                                                    const T2 *__restrict__ D, int N, const double *__restrict__ scale,
                                                    const T *__restrict__ invw) {
  const int H = N / 2 + 1;
  const long long nm = (long long)N * N * H;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += (long long)gridDim.x * blockDim.x) {
    const T2 d = D[m];
    T cc = (T)1;
    if (invw) {
      const int iz = (int)(m % H);
      const long long row = m / H;
      cc = invw[(int)(row / N)] * invw[(int)(row % N)] * invw[iz];
      cc = cc * cc;
    }
    for (int f = 0; f < nf; ++f) {
      T2 *q = F + (long long)f * cslot + m;
      const T2 a = *q;
      const T s = (T)scale[f] * cc;
      T2 r;
      r.x = (a.x * d.x + a.y * d.y) * s;
      r.y = (a.y * d.x - a.x * d.y) * s;
      *q = r;
    }
  }
}

// Two tracers: FA_f <- [sa FA_f conj(DB) + FB_f conj(DA)] s_f W^-2 / 2 for f = 0..nf-1, with FA / FB
// the weighted-field spectra of tracer A / B and DA / DB their density spectra; sa = (-1)^l
// for the Yamamoto fields of odd l (the line of sight through the first galaxy).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) bym_spec_mul_cross(T2 *__restrict__ FA, const T2 *__restrict__ FB,
                                                          long long cslot, int nf, const T2 *__restrict__ DA,
                                                          const T2 *__restrict__ DB, int N,
                                                          const double *__restrict__ scale,
                                                          const T *__restrict__ invw, T sa) {
  const int H = N / 2 + 1;
  const long long nm = (long long)N * N * H;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += (long long)gridDim.x * blockDim.x) {
    const T2 da = DA[m], db = DB[m];
    T cc = (T)0.5;
    if (invw) {
      const int iz = (int)(m % H);
      const long long row = m / H;
      const T w = invw[(int)(row / N)] * invw[(int)(row % N)] * invw[iz];
      cc = (T)0.5 * w * w;
    }
    for (int f = 0; f < nf; ++f) {
      T2 *q = FA + (long long)f * cslot + m;
      const T2 a = *q, b = FB[(long long)f * cslot + m];
      const T s = (T)scale[f] * cc;
      T2 r;
      r.x = (sa * (a.x * db.x + a.y * db.y) + b.x * da.x + b.y * da.y) * s;
      r.y = (sa * (a.y * db.x - a.x * db.y) + b.y * da.x - b.x * da.y) * s;
      *q = r;
    }
  }
}

// The x planes of a padded real slot (N x N x (N + 2)) that hold a non-zero value: one block per
// plane; range[0] <- min, range[1] <- max over them (atomics; the caller sets {N, -1} first).
template <typename T>
__global__ void __launch_bounds__(256) bym_plane_range(const T *__restrict__ d, int N, int *__restrict__ range) {
  const int x = blockIdx.x;
  const long long plane = (long long)N * (N + 2);
  const T *p = d + (long long)x * plane;
  int any = 0;
  for (long long i = threadIdx.x; i < plane; i += blockDim.x) any |= (p[i] != (T)0);
  any = __syncthreads_or(any);
  if (threadIdx.x == 0 && any) {
    atomicMin(range, x);
    atomicMax(range + 1, x);
  }
}

// Interlacing: F_f(k) <- (F_f(k) + P(k) G_f(k)) / 2 for f = 0..nf-1, with G the transform of
// the same field on the mesh shifted by half a cell along each axis and P(k) = prod over the
// axes of ph[n_axis] (per-axis phase exp(-i pi n / N) of the shift, 0 at the Nyquist index).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) bym_interlace(T2 *__restrict__ F, const T2 *__restrict__ G, long long cslot,
                                                     int nf, int N, const T2 *__restrict__ ph) {
  const int H = N / 2 + 1;
  const long long nm = (long long)N * N * H;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(m % H);
    const long long row = m / H;
    const T2 px = ph[(int)(row / N)], py = ph[(int)(row % N)], pz = ph[iz];
    T2 pxy, p;
    pxy.x = px.x * py.x - px.y * py.y;
    pxy.y = px.x * py.y + px.y * py.x;
    p.x = pxy.x * pz.x - pxy.y * pz.y;
    p.y = pxy.x * pz.y + pxy.y * pz.x;
    for (int f = 0; f < nf; ++f) {
      const long long o = (long long)f * cslot + m;
      const T2 a = F[o], b = G[o];
      T2 r;
      r.x = (T)0.5 * (a.x + p.x * b.x - p.y * b.y);
      r.y = (T)0.5 * (a.y + p.x * b.y + p.y * b.x);
      F[o] = r;
    }
  }
}

// ---------------------------------------------------------------- launchers
static unsigned grid_for(long long work, int nsm) {
  long long g = (work + 255) / 256;
  const long long cap = (long long)nsm * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

void launch_norm_reduce(const float4 *p, const float *nbar, long long n, int which, const double lo[3], double inv_h,
                        int N, double *stats, int nsm, cudaStream_t st) {
  if (n <= 0) return;
  bym_norm_reduce<<<grid_for(n, nsm), 256, 0, st>>>(p, nbar, n, which, lo[0], lo[1], lo[2], inv_h, N, stats);
}

template <typename T>
void launch_paint(const float4 *p, long long n, int is_ran, const double *stats, T *delta, int N, const double lo[3],
                  double inv_h, int assign, int nsm, cudaStream_t st, double shift) {
  if (n <= 0) return;
  bym_paint<T><<<grid_for(n, nsm * 4), 256, 0, st>>>(p, n, is_ran, stats, delta, N, lo[0], lo[1], lo[2], inv_h,
                                                      assign, shift);
}

template <typename T, typename T2>
void launch_spec_mul(T2 *F, long long cslot, int nf, const T2 *D, int N, const double *scale, const T *invw, int nsm,
                     cudaStream_t st) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * (N / 2 + 1);
  bym_spec_mul<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(F, cslot, nf, D, N, scale, invw);
}

template <typename T, typename T2>
void launch_spec_mul_cross(T2 *FA, const T2 *FB, long long cslot, int nf, const T2 *DA, const T2 *DB, int N,
                           const double *scale, const T *invw, int nsm, cudaStream_t st, double sa) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * (N / 2 + 1);
  bym_spec_mul_cross<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(FA, FB, cslot, nf, DA, DB, N, scale, invw, (T)sa);
}

template <typename T>
void launch_plane_range(const T *slot, int N, int *range, cudaStream_t st) {
  bym_plane_range<T><<<N, 256, 0, st>>>(slot, N, range);
}

template <typename T, typename T2>
void launch_interlace(T2 *F, const T2 *G, long long cslot, int nf, int N, const T2 *ph, int nsm, cudaStream_t st) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * (N / 2 + 1);
  bym_interlace<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(F, G, cslot, nf, N, ph);
}

template void launch_interlace<float, float2>(float2 *, const float2 *, long long, int, int, const float2 *, int,
                                              cudaStream_t);
template void launch_interlace<double, double2>(double2 *, const double2 *, long long, int, int, const double2 *, int,
                                                cudaStream_t);
template void launch_plane_range<float>(const float *, int, int *, cudaStream_t);
template void launch_plane_range<double>(const double *, int, int *, cudaStream_t);
template void launch_paint<float>(const float4 *, long long, int, const double *, float *, int, const double *, double,
                                  int, int, cudaStream_t, double);
template void launch_paint<double>(const float4 *, long long, int, const double *, double *, int, const double *,
                                   double, int, int, cudaStream_t, double);
template void launch_spec_mul<float, float2>(float2 *, long long, int, const float2 *, int, const double *,
                                             const float *, int, cudaStream_t);
template void launch_spec_mul<double, double2>(double2 *, long long, int, const double2 *, int, const double *,
                                               const double *, int, cudaStream_t);
template void launch_spec_mul_cross<float, float2>(float2 *, const float2 *, long long, int, const float2 *,
                                                   const float2 *, int, const double *, const float *, int,
                                                   cudaStream_t, double);
template void launch_spec_mul_cross<double, double2>(double2 *, const double2 *, long long, int, const double2 *,
                                                     const double2 *, int, const double *, const double *, int,
                                                     cudaStream_t, double);

}  // namespace bym
