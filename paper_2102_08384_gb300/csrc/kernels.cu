// Ahead-of-time kernels of the mesh front end and the spectral products.
//
//   bym_norm_reduce   FP64 sums of w_g, w_r, nbar_r w_r^2 and a count of objects
//                     outside the box (Sec. 2.1: alpha_r and the FKP normalisation);
//   bym_paint_*       CIC / TSC mass assignment of signed weights w and -alpha_r w into the
//                     padded real mesh (periodic, FP64 cell geometry): objects sorted into
//                     tiles, then per-tile fixed-point sums (deterministic, every cell written);
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

constexpr int kPaintTile = 16;
constexpr int kPaintStripes = 16;   // copies of each tile's counter (spreads the atomics of a busy tile)

struct PaintGeom {
  double lo[3], inv_h, shift;         // FP64 geometry (FP64 meshes)
  float lo_h[3], lo_l[3], ih_h, ih_l; // lo and 1/h as float pairs (FP32 meshes)
  float fshift;
  int N, assign, nt;                  // nt = tiles per axis
};

// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// u = (x - lo) inv_h as uh + ul with |ul| <= ulp(uh) / 2
__device__ __forceinline__ void cell_coord(float x, float lo_h, float lo_l, float ih_h, float ih_l, float &uh,
                                           float &ul) {
  float s, e;
  two_sum(x, -lo_h, s, e);                 // x - lo_h = s + e exactly
  const float el = e - lo_l;               // x - lo = s + el (to the rounding of el)
  const float p = s * ih_h;
  const float pe = fmaf(s, ih_h, -p);      // s ih_h = p + pe exactly
  const float q = pe + fmaf(s, ih_l, el * ih_h);
  uh = p + q;                              // renormalise
  ul = q - (uh - p);
}

__device__ __forceinline__ bool in_box(float uh, float ul, int N) {
  return (uh > 0.f || (uh == 0.f && ul >= 0.f)) && (uh < (float)N || (uh == (float)N && ul < 0.f));
}

// an object inside [lo, lo + N h) along every axis, decided as the painter decides it
template <typename T>
__device__ __forceinline__ bool inside_box(const float4 q, const PaintGeom &g) {
  if (sizeof(T) == 4) {
    float uh, ul;
    cell_coord(q.x, g.lo_h[0], g.lo_l[0], g.ih_h, g.ih_l, uh, ul);
    if (!in_box(uh, ul, g.N)) return false;
    cell_coord(q.y, g.lo_h[1], g.lo_l[1], g.ih_h, g.ih_l, uh, ul);
    if (!in_box(uh, ul, g.N)) return false;
    cell_coord(q.z, g.lo_h[2], g.lo_l[2], g.ih_h, g.ih_l, uh, ul);
    return in_box(uh, ul, g.N);
  }
  const double u[3] = {((double)q.x - g.lo[0]) * g.inv_h, ((double)q.y - g.lo[1]) * g.inv_h,
                       ((double)q.z - g.lo[2]) * g.inv_h};
  return u[0] >= 0.0 && u[0] < g.N && u[1] >= 0.0 && u[1] < g.N && u[2] >= 0.0 && u[2] < g.N;
}

struct FF {   // an unevaluated sum of two floats
  float h, l;
};
__device__ __forceinline__ FF ff_add(FF a, float bh, float bl) {
  float s, e;
  two_sum(a.h, bh, s, e);
  e += a.l + bl;
  const float h = s + e;
  return FF{h, e - (h - s)};
}

}  // namespace

// Per-block sums of one catalog (galaxies, which = 0, or randoms, which = 1), written to
// part[5 blockIdx.x + j]: j = 0 sum w, 1 sum nbar w^2 (randoms; nbar may be null: 0), 2 the
// number of objects whose position is not finite or lies outside [lo, lo + N h), 3 sum w^2
// (the shot-noise level of Sec. 2.1), 4 the largest |w| (the scale of the painted sums).
// bym_norm_finish adds them up in block order (so the totals are the same on every run):
// stats[which] += sum w, stats[2] += sum nbar w^2 (randoms), stats[3] += bad,
// stats[4 + which] += sum w^2, stats[6 + which] = max(stats[6 + which], largest |w|).
template <typename T>
__global__ void __launch_bounds__(256) bym_norm_reduce(const float4 *__restrict__ p, const float *__restrict__ nbar,
                                                       long long n, int which, PaintGeom g,
                                                       double *__restrict__ part) {
  // per thread: float-pair sums (w^2 and nbar w^2 from exact float products), exact counts
  FF fw{0.f, 0.f}, fw2{0.f, 0.f}, fnw2{0.f, 0.f};
  int nbad = 0;
  float wa = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 q = p[i];
    if (!(inside_box<T>(q, g) && isfinite(q.w))) ++nbad;
    const float w = q.w;
    fw = ff_add(fw, w, 0.f);
    const float w2 = w * w, w2e = fmaf(w, w, -w2);
    fw2 = ff_add(fw2, w2, w2e);
    wa = fmaxf(wa, fabsf(w));
    if (which == 1 && nbar) {
      const float nb = nbar[i], t = w2 * nb;
      fnw2 = ff_add(fnw2, t, fmaf(w2, nb, -t) + w2e * nb);
    }
  }
  double sw = (double)fw.h + (double)fw.l, sw2 = (double)fw2.h + (double)fw2.l;
  double snw2 = (double)fnw2.h + (double)fnw2.l, bad = (double)nbad, swa = (double)wa;
  __shared__ double red[5][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  sw = warp_sum(sw);
  snw2 = warp_sum(snw2);
  bad = warp_sum(bad);
  sw2 = warp_sum(sw2);
  for (int o = 16; o > 0; o >>= 1) swa = fmax(swa, __shfl_xor_sync(0xffffffffu, swa, o));
  if (lane == 0) {
    red[0][wid] = sw;
    red[1][wid] = snw2;
    red[2][wid] = bad;
    red[3][wid] = sw2;
    red[4][wid] = swa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0, d = 0, f = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
      d += red[3][w];
      f = fmax(f, red[4][w]);
    }
    double *q = part + 5 * (long long)blockIdx.x;
    q[0] = a;
    q[1] = b;
    q[2] = c;
    q[3] = d;
    q[4] = f;
  }
}

// One warp per total: lane l adds the partials of blocks l, l + 32, .. in order, then a fixed
// butterfly; the order of the additions, hence the total, is the same on every run.
__global__ void __launch_bounds__(160) bym_norm_finish(const double *__restrict__ part, int nblk, int which,
                                                       double *__restrict__ stats) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s = j == 4 ? fmax(s, part[5 * b + j]) : s + part[5 * b + j];
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, s, o);
    s = j == 4 ? fmax(s, t) : s + t;
  }
  if (lane) return;
  if (j == 0) stats[which] += s;
  if (j == 1 && which == 1) stats[2] += s;
  if (j == 2) stats[3] += s;
  if (j == 3) stats[4 + which] += s;
  if (j == 4) stats[6 + which] = fmax(stats[6 + which], s);   // the largest |w|: a maximum, not a sum
}

// ---------------------------------------------------------------- painting
// Deterministic mass assignment:
//   bym_paint_prep    per object: its stencil origin b and fractional offsets d (computed once,
//                     so that every later pass sees the same values) and its signed weight (+w
//                     for galaxies, -alpha_r w for randoms) into a record; one count per tile of
//                     kPaintTile^3 cells that its CIC / TSC stencil reaches (an object near a tile
//                     face counts for both tiles, at most 2 per axis);
//   bym_paint_scan_*  exclusive prefix sums of the counts in three parallel phases (per block,
//                     over the block totals, back to every count): the start of each tile's list;
//   bym_paint_fill    each object's index into the lists of its tiles;
//   bym_paint_tile    one CTA per tile: every contribution w W(x) that lands in the tile is
//                     rounded to an integer multiple of 2^-s and summed in 64-bit shared-memory
//                     atomics; then each cell of the tile (and the row padding of the last z tile)
//                     is written once as sum * 2^-s.
// Integer sums do not depend on the order in which the atomics land, so the painted mesh is the
// same bit for bit on every run; its rounding errors are one per contribution and one per cell
// instead of one per atomic add of a floating sum.  FP32 meshes: s is the largest exponent with
// wmax 2^s < 2^30 (wmax = the largest |signed weight|), so a contribution converts to a 32-bit
// integer and a cell's sum of at most 2^32 contributions stays below 2^63; the quantum is wmax
// 2^-30, far below one FP32 rounding of a cell value.  FP64 meshes: s from (n wmax) 2^s < 2^61 and
// 64-bit conversions.  GB300's FP64 pipe is narrow, so in FP32 builds the origin
// u = (x - lo) / h is formed as an unevaluated pair of floats (about 44 bits) on the FP32 pipes.
namespace {

struct alignas(16) PaintD4 {          // FP64 record: offsets and signed weight
  double x, y, z, w;
};
template <typename T>
struct PaintRec;
template <>
struct PaintRec<float> {
  using type = float4;
};
template <>
struct PaintRec<double> {
  using type = PaintD4;
};

// Stencil origin b and offset d of one axis from u = uh + ul (u in [0, N)), FP32 meshes:
// v = u - shift (+ 1/2 for TSC), b = floor(v), d = v - b in [0, 1) (TSC: minus 1/2).
template <int kA>
__device__ __forceinline__ void axis_origin(float uh, float ul, float fshift, int &b, float &d) {
  float vh, ve;
  two_sum(uh, (kA == 3 ? 0.5f : 0.f) - fshift, vh, ve);
  const float vl = ul + ve;
  float fl = floorf(vh);
  float r = (vh - fl) + vl;
  if (r >= 1.f) {
    fl += 1.f;
    r -= 1.f;
  } else if (r < 0.f) {          // v sits a hair below the node fl: one cell down, unless r + 1 rounds to 1
    const float t = r + 1.f;
    if (t < 1.f) {
      fl -= 1.f;
      r = t;
    } else {
      r = 0.f;
    }
  }
  b = (int)fl;
  d = kA == 3 ? r - 0.5f : r;
}

template <typename T, int kA>
__device__ __forceinline__ bool paint_origin(const float4 q, const PaintGeom &g, int b[3],
                                             typename PaintRec<T>::type &r) {
  if (sizeof(T) == 4) {
    float uh[3], ul[3];
    cell_coord(q.x, g.lo_h[0], g.lo_l[0], g.ih_h, g.ih_l, uh[0], ul[0]);
    cell_coord(q.y, g.lo_h[1], g.lo_l[1], g.ih_h, g.ih_l, uh[1], ul[1]);
    cell_coord(q.z, g.lo_h[2], g.lo_l[2], g.ih_h, g.ih_l, uh[2], ul[2]);
    if (!(in_box(uh[0], ul[0], g.N) && in_box(uh[1], ul[1], g.N) && in_box(uh[2], ul[2], g.N))) return false;
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) axis_origin<kA>(uh[a], ul[a], g.fshift, b[a], d[a]);
    r.x = d[0];
    r.y = d[1];
    r.z = d[2];
  } else {
    const double u[3] = {((double)q.x - g.lo[0]) * g.inv_h, ((double)q.y - g.lo[1]) * g.inv_h,
                         ((double)q.z - g.lo[2]) * g.inv_h};
    if (!(u[0] >= 0.0 && u[0] < g.N && u[1] >= 0.0 && u[1] < g.N && u[2] >= 0.0 && u[2] < g.N)) return false;
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double us = u[a] - g.shift;
      const double fl = kA == 2 ? floor(us) : floor(us + 0.5);
      b[a] = (int)fl;
      d[a] = us - fl;
    }
    r.x = d[0];
    r.y = d[1];
    r.z = d[2];
  }
  return true;
}

__device__ __forceinline__ int wrap_cell(int c, int N) { return c < 0 ? c + N : (c >= N ? c - N : c); }

// Tiles (1 or 2) covered along one axis by the stencil cells b + o, o in [omin, omin + kA).
template <int kA>
__device__ __forceinline__ int axis_tiles(int b, const PaintGeom &g, int t[2]) {
  constexpr int omin = kA == 2 ? 0 : -1;
  t[0] = wrap_cell(b + omin, g.N) / kPaintTile;
  t[1] = wrap_cell(b + omin + kA - 1, g.N) / kPaintTile;
  return t[0] == t[1] ? 1 : 2;
}

// the tile counters an object increments (mode 0) or the list slots it fills (mode 1)
template <int kA, int kMode>
__device__ __forceinline__ void paint_tiles(const short4 ob, const PaintGeom &g, int stripe,
                                            unsigned long long *__restrict__ cursor, unsigned *__restrict__ bucket,
                                            unsigned idx) {
  int tx[2], ty[2], tz[2];
  const int nx = axis_tiles<kA>(ob.x, g, tx), ny = axis_tiles<kA>(ob.y, g, ty), nz = axis_tiles<kA>(ob.z, g, tz);
  for (int a = 0; a < nx; ++a)
    for (int c = 0; c < ny; ++c)
      for (int e = 0; e < nz; ++e) {
        const long long t = (((long long)tx[a] * g.nt + ty[c]) * g.nt + tz[e]) * kPaintStripes + stripe;
        if (kMode == 0)
          atomicAdd(cursor + t, 1ull);
        else
          bucket[atomicAdd(cursor + t, 1ull)] = idx;
      }
}

}  // namespace

// Records and tile counts.  s = global warp index mod S: the counter of a busy tile is split over
// S addresses (the same split in bym_paint_fill).
template <typename T, int kA>
__global__ void __launch_bounds__(256) bym_paint_prep(const float4 *__restrict__ gal, long long ng,
                                                      const float4 *__restrict__ ran, long long nr, PaintGeom g,
                                                      const double *__restrict__ stats, short4 *__restrict__ rb,
                                                      typename PaintRec<T>::type *__restrict__ rd,
                                                      unsigned long long *__restrict__ cursor) {
  const int stripe = (int)((((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) % kPaintStripes);
  const double alpha = nr > 0 ? stats[0] / stats[1] : 0.0;
  const T ralpha = (T)(-alpha);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ng + nr;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 q = i < ng ? gal[i] : ran[i - ng];
    int b[3] = {0, 0, 0};
    typename PaintRec<T>::type r;
    const bool ok = paint_origin<T, kA>(q, g, b, r);
    r.w = i < ng ? (T)q.w : ralpha * (T)q.w;
    const short4 ob = make_short4((short)b[0], (short)b[1], (short)b[2], (short)(ok ? 1 : 0));
    rb[i] = ob;
    rd[i] = r;
    if (ok) paint_tiles<kA, 0>(ob, g, stripe, cursor, nullptr, 0u);
  }
}

template <int kA>
__global__ void __launch_bounds__(256) bym_paint_fill(const short4 *__restrict__ rb, long long n, PaintGeom g,
                                                      unsigned long long *__restrict__ cursor,
                                                      unsigned *__restrict__ bucket) {
  const int stripe = (int)((((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) % kPaintStripes);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const short4 ob = rb[i];
    if (ob.w) paint_tiles<kA, 1>(ob, g, stripe, cursor, bucket, (unsigned)i);
  }
}

// Exclusive scan of cursor[0, n) in place into start (and cursor), three phases over blocks of
// 1024 counts; bsum holds one total per block.
__global__ void __launch_bounds__(1024) bym_paint_scan_blocks(const unsigned long long *__restrict__ cursor,
                                                              unsigned long long *__restrict__ start, long long n,
                                                              unsigned long long *__restrict__ bsum) {
  __shared__ unsigned long long part[1024];
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  const unsigned long long v = i < n ? cursor[i] : 0ull;
  part[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
    const unsigned long long a = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += a;
    __syncthreads();
  }
  if (i < n) start[i] = part[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = part[1023];
}

__global__ void __launch_bounds__(1024) bym_paint_scan_totals(unsigned long long *__restrict__ bsum, int nblk,
                                                              unsigned long long *__restrict__ total) {
  __shared__ unsigned long long part[1024];
  const int per = (nblk + 1023) / 1024, a = threadIdx.x * per, e = min(nblk, a + per);
  unsigned long long s = 0;
  for (int b = a; b < e; ++b) s += bsum[b];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
  for (int b = a; b < e; ++b) {
    const unsigned long long c = bsum[b];
    bsum[b] = run;
    run += c;
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

__global__ void __launch_bounds__(1024) bym_paint_scan_apply(unsigned long long *__restrict__ cursor,
                                                             unsigned long long *__restrict__ start, long long n,
                                                             const unsigned long long *__restrict__ bsum) {
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) {
    const unsigned long long v = start[i] + bsum[blockIdx.x];
    start[i] = v;
    cursor[i] = v;
  }
}

// One CTA per tile; the records give the origin, offsets and signed weight of each object.
template <typename T, int kA>
__global__ void __launch_bounds__(256) bym_paint_tile(const short4 *__restrict__ rb,
                                                      const typename PaintRec<T>::type *__restrict__ rd,
                                                      long long n_obj, PaintGeom g,
                                                      const unsigned long long *__restrict__ start,
                                                      const unsigned *__restrict__ bucket,
                                                      const double *__restrict__ stats, long long nr,
                                                      T *__restrict__ delta) {
  __shared__ long long acc[kPaintTile * kPaintTile * kPaintTile];
  __shared__ T scl[2];
  const long long tile = blockIdx.x;
  const int tz = (int)(tile % g.nt), ty = (int)((tile / g.nt) % g.nt), tx = (int)(tile / ((long long)g.nt * g.nt));
  const int x0 = tx * kPaintTile, y0 = ty * kPaintTile, z0 = tz * kPaintTile;
  const int wx = min(kPaintTile, g.N - x0), wy = min(kPaintTile, g.N - y0), wz = min(kPaintTile, g.N - z0);
  for (int i = threadIdx.x; i < kPaintTile * kPaintTile * kPaintTile; i += blockDim.x) acc[i] = 0;
  if (threadIdx.x == 0) {
    // the fixed-point exponent from the largest |signed weight| (FP32) or the bound n wmax (FP64)
    const double alpha = nr > 0 ? fabs(stats[0] / stats[1]) : 0.0;
    const double wmax = fmax(fabs(stats[6]), nr > 0 ? alpha * fabs(stats[7]) : 0.0);
    const double bound = sizeof(T) == 4 ? wmax : wmax * (double)n_obj;
    int ex = 0, sx = 0;
    if (bound > 0.0 && isfinite(bound)) {
      frexp(bound, &ex);                   // bound < 2^ex
      sx = (sizeof(T) == 4 ? 30 : 61) - ex;
    }
    sx = max(-120, min(120, sx));
    scl[0] = (T)ldexp(1.0, sx);
    scl[1] = (T)ldexp(1.0, -sx);
  }
  __syncthreads();
  const T up = scl[0];
  constexpr int omin = kA == 2 ? 0 : -1;
  const unsigned long long e0 = start[tile * kPaintStripes], e1 = start[(tile + 1) * kPaintStripes];
  for (unsigned long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const unsigned i = bucket[e];
    const short4 ob = rb[i];
    const typename PaintRec<T>::type r = rd[i];
    int lx[kA], ly[kA], lz[kA];
#pragma unroll
    for (int o = 0; o < kA; ++o) {
      lx[o] = wrap_cell(ob.x + omin + o, g.N) - x0;
      ly[o] = wrap_cell(ob.y + omin + o, g.N) - y0;
      lz[o] = wrap_cell(ob.z + omin + o, g.N) - z0;
    }
    T wt[3][kA];
    const T dd[3] = {(T)r.x, (T)r.y, (T)r.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T f = dd[a];
      if (kA == 2) {
        wt[a][0] = (T)1 - f;
        wt[a][1] = f;
      } else {
        wt[a][0] = (T)0.5 * ((T)0.5 - f) * ((T)0.5 - f);
        wt[a][1] = (T)0.75 - f * f;
        wt[a][2] = (T)0.5 * ((T)0.5 + f) * ((T)0.5 + f);
      }
    }
    const T ws = (T)r.w * up;
#pragma unroll
    for (int ox = 0; ox < kA; ++ox) {
      if (lx[ox] < 0 || lx[ox] >= wx) continue;
      const T a0 = ws * wt[0][ox];
#pragma unroll
      for (int oy = 0; oy < kA; ++oy) {
        if (ly[oy] < 0 || ly[oy] >= wy) continue;
        const T a1 = a0 * wt[1][oy];
#pragma unroll
        for (int oz = 0; oz < kA; ++oz) {
          if (lz[oz] < 0 || lz[oz] >= wz) continue;
          const T v = a1 * wt[2][oz];
          const long long q = sizeof(T) == 4 ? (long long)__float2int_rn((float)v) : __double2ll_rn((double)v);
          atomicAdd((unsigned long long *)&acc[(lx[ox] * kPaintTile + ly[oy]) * kPaintTile + lz[oz]],
                    (unsigned long long)q);
        }
      }
    }
  }
  __syncthreads();
  const T down = scl[1];
  const long long row = (long long)(g.N + kRowPad);
  const bool pad = z0 + wz == g.N;   // the last z tile also clears the padding values of its rows
  const int rw = pad ? wz + kRowPad : wz;
  for (int i = threadIdx.x; i < wx * wy * rw; i += blockDim.x) {
    const int lz = i % rw, ly = (i / rw) % wy, lx = i / (rw * wy);
    T v = (T)0;
    if (lz < wz) {
      const long long a = acc[(lx * kPaintTile + ly) * kPaintTile + lz];
      if (a != 0) v = (T)a * down;
    }
    delta[((long long)(x0 + lx) * g.N + (y0 + ly)) * row + z0 + lz] = v;
  }
}

// F_f(k) <- F_f(k) conj(D(k)) scale[f] c(k), f = 0..nf-1 (slots of cslot complex
// values each), c = prod_axis invw^2 (compensation, null: 1).  Like the other elementwise
// spectral kernels it runs over the whole padded layout, padding included (harmless there).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) bym_spec_mul(T2 *__restrict__ F, long long cslot, int nf,
                                                    const T2 *__restrict__ D, int N, const double *__restrict__ scale,
                                                    const T *__restrict__ invw) {
  const int H = (N + kRowPad) / 2;   // complex pitch of a row
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
  const int H = (N + kRowPad) / 2;   // complex pitch of a row
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

// The x planes of a padded real slot (N x N x (N + kRowPad)) that hold a non-zero value, and the
// rows y that do in any plane: one block per plane; range[0] <- min, range[1] <- max of x,
// range[2] <- min, range[3] <- max of y over them (atomics; the caller sets {N, -1, N, -1} first).
template <typename T>
__global__ void __launch_bounds__(256) bym_plane_range(const T *__restrict__ d, int N, int *__restrict__ range) {
  __shared__ int ylo, yhi;
  if (threadIdx.x == 0) {
    ylo = N;
    yhi = -1;
  }
  __syncthreads();
  const int x = blockIdx.x;
  const int row = N + kRowPad;
  const T *p = d + (long long)x * N * row;
  int lo = N, hi = -1;
  // a warp per row at a time: coalesced reads, the row's index known without a division
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int y = threadIdx.x >> 5; y < N; y += nw) {
    const T *r = p + (long long)y * row;
    int any = 0;
    for (int z = lane; z < row; z += 32) any |= (r[z] != (T)0);
    if (__any_sync(0xffffffffu, any)) {
      lo = min(lo, y);
      hi = max(hi, y);
    }
  }
  if (hi >= 0) {
    atomicMin(&ylo, lo);
    atomicMax(&yhi, hi);
  }
  __syncthreads();
  if (threadIdx.x == 0 && yhi >= 0) {
    atomicMin(range, x);
    atomicMax(range + 1, x);
    atomicMin(range + 2, ylo);
    atomicMax(range + 3, yhi);
  }
}

// Interlacing: F_f(k) <- (F_f(k) + P(k) G_f(k)) / 2 for f = 0..nf-1, with G the transform of
// the same field on the mesh shifted by half a cell along each axis and P(k) = prod over the
// axes of ph[n_axis] (per-axis phase exp(-i pi n / N) of the shift, 0 at the Nyquist index).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) bym_interlace(T2 *__restrict__ F, const T2 *__restrict__ G, long long cslot,
                                                     int nf, int N, const T2 *__restrict__ ph) {
  const int H = (N + kRowPad) / 2;   // complex pitch of a row
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

size_t norm_scratch_bytes(int nsm) { return sizeof(double) * 5 * (size_t)nsm * 8; }

static PaintGeom make_geom(const double lo[3], double inv_h, int N, int assign, double shift) {
  PaintGeom g;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = lo[a];
    g.lo_h[a] = (float)lo[a];
    g.lo_l[a] = (float)(lo[a] - (double)g.lo_h[a]);
  }
  g.inv_h = inv_h;
  g.ih_h = (float)inv_h;
  g.ih_l = (float)(inv_h - (double)g.ih_h);
  g.shift = shift;
  g.fshift = (float)shift;
  g.N = N;
  g.assign = assign;
  g.nt = (N + kPaintTile - 1) / kPaintTile;
  return g;
}

void launch_norm_reduce(const float4 *p, const float *nbar, long long n, int which, const double lo[3], double inv_h,
                        int N, double *stats, double *part, int nsm, cudaStream_t st, int precision) {
  if (n <= 0) return;
  const unsigned blocks = grid_for(n, nsm);
  const PaintGeom g = make_geom(lo, inv_h, N, 3, 0.0);
  if (precision == 64)
    bym_norm_reduce<double><<<blocks, 256, 0, st>>>(p, nbar, n, which, g, part);
  else
    bym_norm_reduce<float><<<blocks, 256, 0, st>>>(p, nbar, n, which, g, part);
  bym_norm_finish<<<1, 160, 0, st>>>(part, (int)blocks, which, stats);
}

static long long paint_counters(int N) {
  const long long nt = (N + kPaintTile - 1) / kPaintTile;
  return nt * nt * nt * kPaintStripes;
}

size_t paint_scratch_bytes(int N, long long n_objects) {
  const long long ncnt = paint_counters(N), nblk = (ncnt + 1023) / 1024;
  return sizeof(unsigned long long) * (size_t)(2 * ncnt + 2 + nblk) + sizeof(unsigned) * (size_t)(8 * n_objects) +
         sizeof(short4) * (size_t)n_objects + sizeof(PaintD4) * (size_t)n_objects + 1024;
}

template <typename T>
cudaError_t launch_paint(const float4 *gal, long long ng, const float4 *ran, long long nr, const double *stats,
                         T *delta, int N, const double lo[3], double inv_h, int assign, void *scratch, int nsm,
                         cudaStream_t st, double shift) {
  if (ng < 0 || nr < 0 || ng + nr > 0xffffffffll || (assign != 2 && assign != 3)) return cudaErrorInvalidValue;
  const PaintGeom g = make_geom(lo, inv_h, N, assign, shift);
  const long long ntiles = (long long)g.nt * g.nt * g.nt, ncnt = paint_counters(N), nblk = (ncnt + 1023) / 1024;
  const long long n = ng + nr;
  // scratch: cursor[ncnt] | start[ncnt + 1] | bsum[nblk] | records (PaintD4 / float4) | short4 | bucket
  unsigned long long *cursor = (unsigned long long *)scratch, *start = cursor + ncnt, *bsum = start + ncnt + 1;
  char *p = (char *)(bsum + nblk);
  p = (char *)(((unsigned long long)p + 31ull) & ~31ull);
  typename PaintRec<T>::type *rd = (typename PaintRec<T>::type *)p;
  short4 *rb = (short4 *)(p + sizeof(typename PaintRec<T>::type) * (size_t)n);
  unsigned *bucket = (unsigned *)(rb + n);
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long) * (size_t)ncnt, st);
  if (e != cudaSuccess) return e;
  const unsigned gp = grid_for(n, nsm * 4);
  if (n > 0) {
    if (assign == 2)
      bym_paint_prep<T, 2><<<gp, 256, 0, st>>>(gal, ng, ran, nr, g, stats, rb, rd, cursor);
    else
      bym_paint_prep<T, 3><<<gp, 256, 0, st>>>(gal, ng, ran, nr, g, stats, rb, rd, cursor);
  }
  bym_paint_scan_blocks<<<(unsigned)nblk, 1024, 0, st>>>(cursor, start, ncnt, bsum);
  bym_paint_scan_totals<<<1, 1024, 0, st>>>(bsum, (int)nblk, start + ncnt);
  bym_paint_scan_apply<<<(unsigned)nblk, 1024, 0, st>>>(cursor, start, ncnt, bsum);
  if (n > 0) {
    if (assign == 2)
      bym_paint_fill<2><<<gp, 256, 0, st>>>(rb, n, g, cursor, bucket);
    else
      bym_paint_fill<3><<<gp, 256, 0, st>>>(rb, n, g, cursor, bucket);
  }
  if (assign == 2)
    bym_paint_tile<T, 2><<<(unsigned)ntiles, 256, 0, st>>>(rb, rd, n, g, start, bucket, stats, nr, delta);
  else
    bym_paint_tile<T, 3><<<(unsigned)ntiles, 256, 0, st>>>(rb, rd, n, g, start, bucket, stats, nr, delta);
  return cudaGetLastError();
}

template <typename T, typename T2>
void launch_spec_mul(T2 *F, long long cslot, int nf, const T2 *D, int N, const double *scale, const T *invw, int nsm,
                     cudaStream_t st) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * ((N + kRowPad) / 2);
  bym_spec_mul<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(F, cslot, nf, D, N, scale, invw);
}

template <typename T, typename T2>
void launch_spec_mul_cross(T2 *FA, const T2 *FB, long long cslot, int nf, const T2 *DA, const T2 *DB, int N,
                           const double *scale, const T *invw, int nsm, cudaStream_t st, double sa) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * ((N + kRowPad) / 2);
  bym_spec_mul_cross<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(FA, FB, cslot, nf, DA, DB, N, scale, invw, (T)sa);
}

template <typename T>
void launch_plane_range(const T *slot, int N, int *range, cudaStream_t st) {
  bym_plane_range<T><<<N, 256, 0, st>>>(slot, N, range);
}

template <typename T, typename T2>
void launch_interlace(T2 *F, const T2 *G, long long cslot, int nf, int N, const T2 *ph, int nsm, cudaStream_t st) {
  if (nf <= 0) return;
  const long long nm = (long long)N * N * ((N + kRowPad) / 2);
  bym_interlace<T, T2><<<grid_for(nm, nsm), 256, 0, st>>>(F, G, cslot, nf, N, ph);
}

template void launch_interlace<float, float2>(float2 *, const float2 *, long long, int, int, const float2 *, int,
                                              cudaStream_t);
template void launch_interlace<double, double2>(double2 *, const double2 *, long long, int, int, const double2 *, int,
                                                cudaStream_t);
template void launch_plane_range<float>(const float *, int, int *, cudaStream_t);
template void launch_plane_range<double>(const double *, int, int *, cudaStream_t);
template cudaError_t launch_paint<float>(const float4 *, long long, const float4 *, long long, const double *, float *,
                                         int, const double *, double, int, void *, int, cudaStream_t, double);
template cudaError_t launch_paint<double>(const float4 *, long long, const float4 *, long long, const double *,
                                          double *, int, const double *, double, int, void *, int, cudaStream_t,
                                          double);
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
