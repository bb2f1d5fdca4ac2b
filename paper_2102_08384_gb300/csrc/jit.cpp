// Kernel generator for the field-dependent steps of the estimators.
//
// For one (LOS, ell_max, order K, precision) it writes a CUDA C++ module with
//   gen_fields   field generation: Y_{J nu}(hat x) (2r/r0)^-alpha delta(x) for every
//                field the series needs, one pass over the mesh (FP64 recurrence);
//   kgeom/rgeom  mode / lag-cell counts and mean |k| / |Delta| per shell;
//   kcontract    k-space contraction with Y_{l mu}(hat k) and FP64 shell sums
//                (Yamamoto: Re F conj(delta); midpoint: Re F[H]; bisector: the
//                bilinear form sum B Re(conj F_i F_j));
//   kcontract_x  bisector variant that also writes X_{l mu}(k) for the xi path;
//   mid_combine  midpoint Delta-space combine H_{l mu} = sum phi Y (|Delta|/r0)^alpha g;
//   xi_lag       configuration-space contraction over the lag cube r < r_max.
// The couplings (phi, B, f) enter as floating-point immediates and every
// field value lives in a register, so the sparse sums compile to plain FMA
// streams.  Real spherical harmonics are produced by an unrolled
// associated-Legendre recurrence (orthonormal, no Condon-Shortley phase).
#include "jit.h"

#include <nvrtc.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <set>
#include <sstream>

#include "coeff.h"

namespace bym {
namespace {

std::string lit(double v, bool f32) {
  char buf[64];
  if (f32)
    snprintf(buf, sizeof buf, "(%.9ef)", v);
  else
    snprintf(buf, sizeof buf, "(%.17e)", v);
  return buf;
}

// Declares variables P<l*l+l+nu> = Y_{l nu}(u) for l <= L from the unit vector
// (ux, uy, uz); zm (0 or 1) zeroes every l > 0 term (the zero vector carries
// Y = delta_{l0} / sqrt(4 pi)).  Y_{l, +-m} = sqrt2 p_l^m(uz) Re / Im (ux + i uy)^m with p_l^m the
// normalised associated-Legendre polynomial without its sin^m factor.  az32 (FP64 build of the
// recurrence only): the recurrence over l runs in FP64, the azimuthal factor (ux + i uy)^m and
// the products in FP32, and P<..> are floats.
void emit_ylm(std::ostream &o, int L, bool f32, const std::string &P, const std::string &ux,
              const std::string &uy, const std::string &uz, const std::string &zm, bool az32 = false) {
  const char *TY = f32 ? "float" : "double";
  const char *TA = f32 || az32 ? "float" : "double";   // the azimuthal factor and the products
  const std::string ax = az32 ? "(float)" + ux : ux, ay = az32 ? "(float)" + uy : uy;
  o << "  " << TA << " " << P << "c0 = 1, " << P << "s0 = 0;\n";
  for (int m = 1; m <= L; ++m)
    o << "  " << TA << " " << P << "c" << m << " = " << P << "c" << m - 1 << " * " << ax << " - " << P << "s"
      << m - 1 << " * " << ay << ", " << P << "s" << m << " = " << P << "s" << m - 1 << " * " << ax << " + " << P
      << "c" << m - 1 << " * " << ay << ";\n";
  for (int m = 0; m <= L; ++m) {
    if (m == 0)
      o << "  " << TY << " " << P << "p0_0 = " << lit(1.0 / std::sqrt(4.0 * M_PI), f32) << ";\n";
    else
      o << "  " << TY << " " << P << "p" << m << "_" << m << " = " << P << "p" << m - 1 << "_" << m - 1 << " * "
        << lit(std::sqrt((2.0 * m + 1) / (2.0 * m)), f32) << ";\n";
    if (m + 1 <= L)
      o << "  " << TY << " " << P << "p" << m + 1 << "_" << m << " = " << lit(std::sqrt(2.0 * m + 3), f32) << " * "
        << uz << " * " << P << "p" << m << "_" << m << ";\n";
    for (int l = m + 2; l <= L; ++l) {
      const double a = std::sqrt((4.0 * l * l - 1) / ((double)l * l - (double)m * m));
      const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1));
      o << "  " << TY << " " << P << "p" << l << "_" << m << " = " << lit(a, f32) << " * (" << uz << " * " << P
        << "p" << l - 1 << "_" << m << " - " << lit(b, f32) << " * " << P << "p" << l - 2 << "_" << m << ");\n";
    }
    for (int l = m; l <= L; ++l) {
      if (m == 0) {
        o << "  " << TA << " " << P << l * l + l << " = " << (az32 ? "(float)(" : "(") << P << "p" << l << "_0";
        if (l > 0) o << " * " << zm;
        o << ");\n";
      } else {
        // sqrt2 p_l^m once (in the recurrence's precision), then the azimuthal products
        const std::string q = az32 ? "(float)(" + lit(std::sqrt(2.0), false) + " * " + P + "p" + std::to_string(l) +
                                         "_" + std::to_string(m) + ")"
                                   : lit(std::sqrt(2.0), f32) + " * " + P + "p" + std::to_string(l) + "_" +
                                         std::to_string(m);
        o << "  " << TA << " " << P << l * l + l + m << " = " << q << " * " << P << "c" << m << ";\n";
        o << "  " << TA << " " << P << l * l + l - m << " = " << q << " * " << P << "s" << m << ";\n";
      }
    }
  }
}

const char *kPrelude = R"(
#define BYM_FULL 0xffffffffu
template <typename V>
__device__ __forceinline__ V bym_wsum(V v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(BYM_FULL, v, o);
  return v;
}
// FP64 shell sums of n = nbins * NL values.  Every lane holds (bin, v[NL]); lanes that share a bin
// are pre-reduced with shuffles (a fixed butterfly) and the group leader adds the partial sum to a
// shared accumulator.  With dynamic shared memory for one accumulator per warp (8 n doubles; 256
// threads) each warp adds into its own in the order of its bins, the block adds the 8 in warp order,
// every block writes its totals after the n sums in global memory (g[n] is a ticket counter,
// g[n + 1 + b n + i] block b's total of sum i), and the last block to finish adds them in block
// order: the sums are then the same on every run.  With room for one accumulator the warps share it
// through atomics, which orders the additions by arrival.
__device__ __forceinline__ int bym_nacc(int n) {
  unsigned sz;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(sz));
  return sz >= 64u * (unsigned)n ? 8 : 1;
}
template <int NL, typename V>
__device__ __forceinline__ void bym_bin_flush(int bin, const V (&v)[NL], double *s, int n) {
  const bool own = bym_nacc(n) == 8;
  double *sw = own ? s + (threadIdx.x >> 5) * n : s;
  unsigned pending = __ballot_sync(BYM_FULL, bin >= 0);
  const int lane = threadIdx.x & 31;
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int bl = __shfl_sync(BYM_FULL, bin, leader);
    const bool mine = (bin == bl);
    const unsigned grp = __ballot_sync(BYM_FULL, mine);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const V x = bym_wsum<V>(mine ? v[l] : (V)0);
      if (lane == leader) {
        if (own)
          sw[bl * NL + l] += (double)x;
        else
          atomicAdd(sw + bl * NL + l, (double)x);
      }
    }
    pending &= ~grp;
  }
}
__device__ __forceinline__ void bym_bins_init(double *s, int n) {
  const int m = bym_nacc(n) * n;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = 0.0;
  __syncthreads();
}
__device__ __forceinline__ void bym_bins_out(const double *s, double *g, int n) {
  __shared__ int bym_last;
  __syncthreads();
  const int nacc = bym_nacc(n);
  double *part = g + n + 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = 0.0;
    for (int w = 0; w < nacc; ++w) x += s[w * n + i];
    part[(long long)blockIdx.x * n + i] = x;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    bym_last = atomicAdd((unsigned long long *)(g + n), 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!bym_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) x += __ldcg(part + (long long)b * n + i);
    g[i] += x;
  }
  if (threadIdx.x == 0) *(unsigned long long *)(g + n) = 0ull;
}
__device__ __forceinline__ int bym_lab(int i, int N) { return i < N / 2 ? i : i - N; }
__device__ __forceinline__ float bym_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double bym_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float bym_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double bym_sqrt(double x) { return sqrt(x); }
)";

struct Fields {
  std::vector<FieldInfo> list;
};

Fields field_set(const JitKey &k) {
  Fields f;
  if (k.los == 0) {  // Yamamoto: Y_{l mu} delta, even l
    for (int l = 0; l <= k.ell_max; l += 2)
      for (int nu = -l; nu <= l; ++nu) f.list.push_back({0, l, nu});
  } else if (k.los == 2) {  // bisector: Y_{J nu} delta, J <= ell_max + floor(K/2)
    const int Jmax = k.ell_max + k.K / 2;
    for (int J = 0; J <= Jmax; ++J)
      for (int nu = -J; nu <= J; ++nu) f.list.push_back({0, J, nu});
  } else {  // midpoint (all-parity, or even alpha only for the parity-even form): g^alpha_{J nu}
    for (auto &g : midpoint_gfields(k.ell_max, k.K, k.los == 3)) f.list.push_back({g.alpha, g.J, g.nu});
  }
  return f;
}

void emit_bin_loop_head(std::ostream &o, const std::string &count_expr) {
  o << "  const int lane = threadIdx.x & 31;\n";
  o << "  const long long total = " << count_expr << ";\n";
  o << "  for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < total;"
       " base += (long long)gridDim.x * blockDim.x) {\n";
  o << "    const long long m = base + lane;\n";
}

// gen_fields kernel for fields [f0, f1) of the list, written to slots 0 .. f1 - f0 of out.
// f32: FP32 build (the azimuthal factor and the products in FP32, the Legendre recurrence in FP64).
void emit_gen_fields(std::ostream &o, const char *name, const std::vector<FieldInfo> &list, int f0, int f1,
                     bool f32) {
  int Jmax = 0, amax = 0;
  for (int i = f0; i < f1; ++i) {
    Jmax = std::max(Jmax, list[i].J);
    amax = std::max(amax, list[i].alpha);
  }
  // one thread per value of the padded rows y in [y0, y0 + ny) of the x planes [x0, x0 + np):
  // every value of those rows of every field is written (zero where delta is zero and in the row
  // padding), so the field slots need no zero-fill; a warp stores 32 consecutive values of a row
  // per field
  o << "extern \"C\" __global__ void __launch_bounds__(256, 2) " << name << "(const real* __restrict__ delta,"
       " real* __restrict__ out, long long slot, int N, double lo0, double lo1, double lo2, double h,"
       " double inv_r0, int x0, int np, int y0, int ny) {\n";
  o << "  const long long row = N + 4;\n";
  o << "  const long long nval = (long long)np * ny * row;\n";
  o << "  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nval;"
       " c += (long long)gridDim.x * blockDim.x) {\n";
  o << "    const int iz = (int)(c % row); const long long t = c / row;\n";
  o << "    const int iy = y0 + (int)(t % ny); const int ix = x0 + (int)(t / ny);\n";
  o << "    const long long off = ((long long)ix * N + iy) * row + iz;\n";
  o << "    const real d = iz < N ? delta[off] : (real)0;\n";
  o << "    if (d == (real)0) {\n";
  for (int i = f0; i < f1; ++i) o << "      out[" << i - f0 << "LL * slot + off] = (real)0;\n";
  o << "      continue;\n    }\n";
  o << "    const double x = lo0 + ix * h, y = lo1 + iy * h, z = lo2 + iz * h;\n";
  o << "    const double r2 = x * x + y * y + z * z;\n";
  o << "    const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;\n";
  o << "    const double ux = x * ir, uy = y * ir, uz = z * ir, zm = r2 > 0.0 ? 1.0 : 0.0;\n";
  o << "    const double rad0 = (double)d;\n";
  if (amax > 0) o << "    const double q = r2 > 0.0 ? 1.0 / (2.0 * sqrt(r2) * inv_r0) : 0.0;\n";
  for (int a = 1; a <= amax; ++a) o << "    const double rad" << a << " = rad" << a - 1 << " * q;\n";
  for (int a = 0; a <= amax; ++a) o << "    const real rr" << a << " = (real)rad" << a << ";\n";
  emit_ylm(o, Jmax, false, "y", "ux", "uy", "uz", "zm", f32);
  for (int i = f0; i < f1; ++i)
    o << "    out[" << i - f0 << "LL * slot + off] = (real)y" << ylm_index(list[i].J, list[i].nu) << " * rr"
      << list[i].alpha << ";\n";
  o << "  }\n}\n";
}

// mid_combine for the g fields [f0, f1) (read from slots 0 .. f1 - f0 of G): H = (or +=) the
// terms of H_{l mu} = sum phi Y (|Delta|/r0)^alpha g that involve those fields.
void emit_mid_combine(std::ostream &o, const char *name, const JitKey &key, const std::vector<MidTerm> &terms,
                      int f0, int f1, bool accumulate, int n_out = -1) {
  const bool f32 = key.prec == 32;
  const int n_lm = n_out >= 0 ? n_out : n_even_lm(key.ell_max);
  o << "extern \"C\" __global__ void __launch_bounds__(256) " << name << "(const real* __restrict__ G,"
       " long long slot, real* __restrict__ Hout, int N, double tscale) {\n";
  o << "  const long long ncell = (long long)N * N * N;\n";
  o << "  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;"
       " c += (long long)gridDim.x * blockDim.x) {\n";
  o << "    const int iz = (int)(c % N); const long long t = c / N;\n";
  o << "    const int iy = (int)(t % N); const int ix = (int)(t / N);\n";
  o << "    const long long off = ((long long)ix * N + iy) * (N + 4) + iz;\n";
  o << "    const int jx = bym_lab(ix, N), jy = bym_lab(iy, N), jz = bym_lab(iz, N);\n";
  o << "    const int j2 = jx * jx + jy * jy + jz * jz;\n";
  o << "    const real rr = bym_sqrt((real)j2);\n";
  o << "    const real ir = j2 > 0 ? (real)1 / rr : (real)0;\n";
  o << "    const real ux = jx * ir, uy = jy * ir, uz = jz * ir, zm = j2 > 0 ? (real)1 : (real)0;\n";
  o << "    const real t1 = (real)(rr * tscale);\n";
  for (int a = 2; a <= key.K; ++a) o << "    const real t" << a << " = t" << a - 1 << " * t1;\n";
  {
    std::ostringstream yy;
    emit_ylm(yy, key.K, f32, "yd", "ux", "uy", "uz", "zm");
    std::istringstream is(yy.str());
    std::string line;
    while (std::getline(is, line)) o << "  " << line << "\n";
  }
  std::set<int> touched;
  for (auto &tm : terms)
    if (tm.g >= f0 && tm.g < f1) touched.insert(tm.lm);
  for (int i = 0; i < n_lm; ++i) o << "    real H" << i << " = (real)0;\n";
  for (int a = 0; a <= key.K; ++a) {
    std::set<int> gs;
    std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> groups;  // (lm, y) -> (g, c)
    for (auto &tm : terms)
      if (tm.alpha == a && tm.g >= f0 && tm.g < f1) {
        gs.insert(tm.g);
        groups[{tm.lm, tm.y}].push_back({tm.g, tm.c});
      }
    if (groups.empty()) continue;
    o << "    {\n";
    for (int g : gs) o << "      const real g" << g << " = G[" << g - f0 << "LL * slot + off];\n";
    for (auto &kv : groups) {
      o << "      { real S = (real)0;";
      for (auto &gc : kv.second) o << " S += " << lit(gc.second, f32) << " * g" << gc.first << ";";
      o << " H" << kv.first.first << " += yd" << kv.first.second;
      if (a > 0) o << " * t" << a;
      o << " * S; }\n";
    }
    o << "    }\n";
  }
  for (int i = 0; i < n_lm; ++i) {
    if (!accumulate)
      o << "    Hout[" << i << "LL * slot + off] = H" << i << ";\n";
    else if (touched.count(i))
      o << "    Hout[" << i << "LL * slot + off] += H" << i << ";\n";
  }
  o << "  }\n}\n";
}

// xi_lag: the configuration-space contraction over the lag cube.  For the
// midpoint forms only the g fields [f0, f1) enter (read from slots 0 .. f1 - f0
// of Z), so a field range adds its share of the shell sums.  Returns the
// harmonic degree needed on the lag grid.
int emit_xi_lag(std::ostream &o, const char *name, const JitKey &key, int f0, int f1) {
  const int L = key.ell_max, NL = L / 2 + 1;
  const bool midpoint = key.los == 1 || key.los == 3, even = key.los == 3;
  int jlag = L;
  std::vector<XiTerm> xterms;
  if (midpoint) {
    xterms = midpoint_xi_terms(key.ell_max, key.K, even);
    for (auto &x : xterms) jlag = std::max(jlag, x.J);
  }
  o << "extern \"C\" __global__ void __launch_bounds__(256) " << name << "(const real* __restrict__ Z, long long slot,"
       " int N, int jm, int full, const int* __restrict__ lut, int nbins, double* __restrict__ gsum,"
       " double zscale, double tscale) {\n";
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * " << NL << ");\n";
  o << "  const int Lc = full ? N : 2 * jm + 1;\n";
  emit_bin_loop_head(o, "(long long)Lc * Lc * Lc");
  o << "    int bin = -1; double v[" << NL << "] = {";
  for (int l = 0; l < NL; ++l) o << (l ? ", " : "") << "0.0";
  o << "};\n";
  o << "    if (m < total) {\n";
  o << "      const int a = (int)(m % Lc); const long long t = m / Lc;\n";
  o << "      const int b = (int)(t % Lc); const int c = (int)(t / Lc);\n";
  o << "      const int jx = full ? bym_lab(c, N) : c - jm, jy = full ? bym_lab(b, N) : b - jm,"
       " jz = full ? bym_lab(a, N) : a - jm;\n";
  o << "      const int j2 = jx * jx + jy * jy + jz * jz;\n";
  o << "      bin = lut[j2];\n";
  o << "      if (bin >= 0) {\n";
  o << "        const int ix = jx < 0 ? jx + N : jx, iy = jy < 0 ? jy + N : jy, iz = jz < 0 ? jz + N : jz;\n";
  o << "        const long long off = ((long long)ix * N + iy) * (N + 4) + iz;\n";
  o << "        const double rr = sqrt((double)j2); const double ir = 1.0 / rr;\n";
  o << "        const double ux = jx * ir, uy = jy * ir, uz = jz * ir, zm = 1.0;\n";
  {
    std::ostringstream yy;
    emit_ylm(yy, jlag, false, "yl", "ux", "uy", "uz", "zm");
    std::istringstream is(yy.str());
    std::string line;
    while (std::getline(is, line)) o << "      " << line << "\n";
  }
  if (midpoint) {
    int amax = 0;
    for (auto &x : xterms) amax = std::max(amax, x.alpha);
    o << "        const double t1 = rr * tscale;\n";
    for (int a2 = 2; a2 <= amax; ++a2) o << "        const double t" << a2 << " = t" << a2 - 1 << " * t1;\n";
    for (int l = 0; l <= L; l += 2) {
      o << "        { double T = 0.0;\n";
      for (auto &x : xterms) {
        if (x.l != l) continue;
        std::ostringstream sum;
        for (int nu = -x.J; nu <= x.J; ++nu) {
          const int g = midpoint_gfield_index(key.ell_max, x.alpha, x.J, nu, even);
          if (g >= f0 && g < f1)
            sum << " S += yl" << ylm_index(x.J, nu) << " * (double)Z[" << g - f0 << "LL * slot + off];";
        }
        if (sum.str().empty()) continue;
        o << "          { double S = 0.0;" << sum.str() << " T += " << lit(x.f, false);
        if (x.alpha > 0) o << " * t" << x.alpha;
        o << " * S; }\n";
      }
      o << "          v[" << l / 2 << "] = T * zscale; }\n";
    }
  } else {
    for (int l = 0; l <= L; l += 2) {
      o << "        { double T = 0.0;";
      for (int mu = -l; mu <= l; ++mu)
        o << " T += yl" << ylm_index(l, mu) << " * (double)Z[" << even_lm_index(l, mu) << "LL * slot + off];";
      o << " v[" << l / 2 << "] = T * zscale; }\n";
    }
  }
  o << "      }\n    }\n";
  o << "    bym_bin_flush<" << NL << ", double>(bin, v, s, nbins * " << NL << ");\n  }\n  bym_bins_out(s, gsum, nbins * " << NL << ");\n}\n";
  return jlag;
}

// Bisector contraction for the field pairs (i, j), i <= j, with i in [a0, a1) read
// from FA and j in [b0, b1) read from FB (slot i - a0, j - b0): adds that share of
// X_{lm}(k) = sum c Re(conj F_i F_j) to the P shell sums and, when xout is given,
// writes (accumulate = 0) or adds (accumulate = 1) it to X_{lm}(k).
// cross: two tracers, FA = F[Y_i delta_A], FB = F[Y_j delta_B] (every field of each);
// each symmetrised term c (i < j) splits into c/2 on (i, j) and c/2 on (j, i), so that
// X_{lm}(k) = sum over ordered pairs of c_ij Re(conj F^A_i F^B_j): the Hermitian part of
// the bilinear sum of eq. bisector-pk-fft with delta_A at r_1 and delta_B at r_2.
void emit_kcontract_pair(std::ostream &o, const char *name, const JitKey &key, int a0, int a1, int b0, int b1,
                         bool cross = false) {
  const bool f32 = key.prec == 32;
  const int L = key.ell_max, NL = L / 2 + 1, n_lm = n_even_lm(L);
  o << "extern \"C\" __global__ void __launch_bounds__(256) " << name
    << "(const real2* __restrict__ FA, const real2* __restrict__ FB, long long cslot, int N,"
       " const int* __restrict__ lut, int nbins, double* __restrict__ gsum, real2* __restrict__ xout,"
       " long long xslot, const real* __restrict__ invw, int accumulate) {\n";
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * " << NL << ");\n  const int H = N / 2 + 1;\n";
  emit_bin_loop_head(o, "(long long)N * N * H");
  o << "    int bin = -1; double v[" << NL << "] = {";
  for (int l = 0; l < NL; ++l) o << (l ? ", " : "") << "0.0";
  o << "};\n";
  o << "    if (m < total) {\n";
  o << "      const int iz = (int)(m % H); const long long row = m / H, mo = row * (H + 1) + iz;\n";
  o << "      const int ix = (int)(row / N), iy = (int)(row % N);\n";
  o << "      const int nx = bym_lab(ix, N), ny = bym_lab(iy, N), nz = (iz == N / 2) ? -N / 2 : iz;\n";
  o << "      const int n2 = nx * nx + ny * ny + nz * nz;\n";
  o << "      bin = lut[n2];\n";
  o << "      if (xout || bin >= 0) {\n";
  o << "        real cc = (real)1;\n";
  o << "        if (invw) { cc = invw[ix] * invw[iy] * invw[iz]; cc = cc * cc; }\n";
  for (int i = 0; i < n_lm; ++i) o << "        real X" << i << " = (real)0;\n";
  std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> by_pair;
  for (auto &t : bisector_terms(key.ell_max, key.K)) {
    if (cross) {
      if (t.i == t.j) {
        by_pair[{t.i, t.j}].push_back({t.lm, t.c});
      } else {
        by_pair[{t.i, t.j}].push_back({t.lm, 0.5 * t.c});
        by_pair[{t.j, t.i}].push_back({t.lm, 0.5 * t.c});
      }
    } else if (t.i >= a0 && t.i < a1 && t.j >= b0 && t.j < b1) {
      by_pair[{t.i, t.j}].push_back({t.lm, t.c});
    }
  }
  std::set<int> ua, ub;
  for (auto &kv : by_pair) {
    ua.insert(kv.first.first);
    ub.insert(kv.first.second);
  }
  const bool same = !cross && a0 == b0;
  const char *na = cross ? "a" : "f", *nb = cross ? "b" : "f";
  // cross: B's fields first, then each A field just before the terms that use it
  if (!cross)
    for (int i : ua) o << "        const real2 f" << i << " = FA[" << i - a0 << "LL * cslot + mo];\n";
  for (int j : ub)
    if (!(same && ua.count(j)))
      o << "        const real2 " << nb << j << " = " << (same ? "FA[" : "FB[") << j - b0 << "LL * cslot + mo];\n";
  int cur = -1;
  for (auto &kv : by_pair) {
    const int i = kv.first.first, j = kv.first.second;
    if (cross && i != cur) {
      if (cur >= 0) o << "        }\n";
      o << "        { const real2 a" << i << " = FA[" << i - a0 << "LL * cslot + mo];\n";
      cur = i;
    }
    o << "        { const real q = " << na << i << ".x * " << nb << j << ".x + " << na << i << ".y * " << nb << j
      << ".y;";
    for (auto &lc : kv.second) o << " X" << lc.first << " += " << lit(lc.second, f32) << " * q;";
    o << " }\n";
  }
  if (cross && cur >= 0) o << "        }\n";
  for (int i = 0; i < n_lm; ++i) o << "        X" << i << " *= cc;\n";
  o << "        if (xout) {\n";
  for (int i = 0; i < n_lm; ++i)
    o << "          { real2 xv; xv.x = X" << i << " + (accumulate ? xout[" << i << "LL * xslot + mo].x : (real)0);"
      << " xv.y = (real)0; xout[" << i << "LL * xslot + mo] = xv; }\n";
  o << "        }\n";
  o << "        if (bin >= 0) {\n";
  o << "          const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;\n";
  o << "          const double r2 = (double)n2; const double ir = bym_rsqrt(r2);\n";
  o << "          const double ux = nx * ir, uy = ny * ir, uz = nz * ir; const double zm = 1.0;\n";
  {
    std::ostringstream yy;
    emit_ylm(yy, L, false, "yk", "ux", "uy", "uz", "zm", f32);
    std::istringstream is(yy.str());
    std::string line;
    while (std::getline(is, line)) o << "        " << line << "\n";
  }
  for (int l = 0; l <= L; l += 2) {
    o << "          { double T = 0.0;";
    for (int mu = -l; mu <= l; ++mu) o << " T += yk" << ylm_index(l, mu) << " * (double)X" << even_lm_index(l, mu) << ";";
    o << " v[" << l / 2 << "] = w * T; }\n";
  }
  o << "        }\n      }\n    }\n";
  o << "    bym_bin_flush<" << NL << ", double>(bin, v, s, nbins * " << NL << ");\n  }\n  bym_bins_out(s, gsum, nbins * " << NL << ");\n}\n";
}

}  // namespace

std::string generate_source(const JitKey &key, KernelSet *meta) {
  const bool f32 = key.prec == 32;
  const char *real = f32 ? "float" : "double";
  const int L = key.ell_max;
  const int n_lm = n_even_lm(L);
  const int NL = L / 2 + 1;
  const Fields F = field_set(key);
  const int nf = (int)F.list.size();
  const bool midpoint = key.los == 1 || key.los == 3, even = key.los == 3;
  std::ostringstream o;
  o << "typedef " << real << " real;\ntypedef " << real << "2 real2;\n";
  o << kPrelude;

  // ------------------------------------------------------------------ gen_fields
  emit_gen_fields(o, "gen_fields", F.list, 0, nf, key.prec == 32);

  // ------------------------------------------------------------------ geometry
  o << "extern \"C\" __global__ void __launch_bounds__(256) kgeom(int N, const int* __restrict__ lut, int nbins,"
       " double kf, double* __restrict__ gsum) {\n";
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * 2);\n  const int H = N / 2 + 1;\n";
  emit_bin_loop_head(o, "(long long)N * N * H");
  o << "    int bin = -1; double v[2] = {0.0, 0.0};\n";
  o << "    if (m < total) {\n";
  o << "      const int iz = (int)(m % H); const long long row = m / H, mo = row * (H + 1) + iz;\n";
  o << "      const int nx = bym_lab((int)(row / N), N), ny = bym_lab((int)(row % N), N);\n";
  o << "      const int nz = (iz == N / 2) ? -N / 2 : iz;\n";
  o << "      const int n2 = nx * nx + ny * ny + nz * nz;\n";
  o << "      bin = lut[n2];\n";
  o << "      if (bin >= 0) { const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;"
       " v[0] = w; v[1] = w * kf * sqrt((double)n2); }\n";
  o << "    }\n    bym_bin_flush<2, double>(bin, v, s, nbins * 2);\n  }\n  bym_bins_out(s, gsum, nbins * 2);\n}\n";

  o << "extern \"C\" __global__ void __launch_bounds__(256) rgeom(int N, int jm, int full,"
       " const int* __restrict__ lut, int nbins, double h, double* __restrict__ gsum) {\n";
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * 2);\n";
  o << "  const int Lc = full ? N : 2 * jm + 1;\n";
  emit_bin_loop_head(o, "(long long)Lc * Lc * Lc");
  o << "    int bin = -1; double v[2] = {0.0, 0.0};\n";
  o << "    if (m < total) {\n";
  o << "      const int a = (int)(m % Lc); const long long t = m / Lc;\n";
  o << "      const int b = (int)(t % Lc); const int c = (int)(t / Lc);\n";
  o << "      const int jx = full ? bym_lab(c, N) : c - jm, jy = full ? bym_lab(b, N) : b - jm,"
       " jz = full ? bym_lab(a, N) : a - jm;\n";
  o << "      const int j2 = jx * jx + jy * jy + jz * jz;\n";
  o << "      bin = lut[j2];\n";
  o << "      if (bin >= 0) { v[0] = 1.0; v[1] = h * sqrt((double)j2); }\n";
  o << "    }\n    bym_bin_flush<2, double>(bin, v, s, nbins * 2);\n  }\n  bym_bins_out(s, gsum, nbins * 2);\n}\n";

  // ------------------------------------------------------------------ k-space contraction
  auto emit_kcontract = [&](const char *name, bool with_x) {
    // the bisector form with X written holds ~140 registers unbounded: two blocks per SM (16 warps)
    o << "extern \"C\" __global__ void __launch_bounds__(256" << (with_x ? ", 2" : "") << ") " << name
      << "(const real2* __restrict__ F, long long cslot, const real2* __restrict__ D, int N,"
         " const int* __restrict__ lut, int nbins, double* __restrict__ gsum, real2* __restrict__ xout,"
         " long long xslot, const real* __restrict__ invw) {\n";
    o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * " << NL << ");\n  const int H = N / 2 + 1;\n";
    emit_bin_loop_head(o, "(long long)N * N * H");
    o << "    int bin = -1; double v[" << NL << "] = {";
    for (int l = 0; l < NL; ++l) o << (l ? ", " : "") << "0.0";
    o << "};\n";
    o << "    if (m < total) {\n";
    o << "      const int iz = (int)(m % H); const long long row = m / H, mo = row * (H + 1) + iz;\n";
    o << "      const int ix = (int)(row / N), iy = (int)(row % N);\n";
    o << "      const int nx = bym_lab(ix, N), ny = bym_lab(iy, N), nz = (iz == N / 2) ? -N / 2 : iz;\n";
    o << "      const int n2 = nx * nx + ny * ny + nz * nz;\n";
    o << "      bin = lut[n2];\n";
    o << "      if (" << (with_x ? "true" : "bin >= 0") << ") {\n";
    o << "        real cc = (real)1;\n";
    if (!midpoint)
      o << "        if (invw) { cc = invw[ix] * invw[iy] * invw[iz]; cc = cc * cc; }\n";
    // X_{lm}
    for (int i = 0; i < n_lm; ++i) o << "        real X" << i << " = (real)0;\n";
    if (key.los == 0) {
      o << "        const real2 d = D[mo];\n";
      for (int i = 0; i < n_lm; ++i)
        o << "        { const real2 f = F[" << i << "LL * cslot + mo]; X" << i << " = (f.x * d.x + f.y * d.y) * cc; }\n";
    } else if (midpoint) {
      for (int i = 0; i < n_lm; ++i) o << "        X" << i << " = F[" << i << "LL * cslot + mo].x;\n";
    } else {
      for (int i = 0; i < nf; ++i) o << "        const real2 f" << i << " = F[" << i << "LL * cslot + mo];\n";
      auto terms = bisector_terms(key.ell_max, key.K);
      std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> by_pair;
      for (auto &t : terms) by_pair[{t.i, t.j}].push_back({t.lm, t.c});
      for (auto &kv : by_pair) {
        const int i = kv.first.first, j = kv.first.second;
        o << "        { const real q = f" << i << ".x * f" << j << ".x + f" << i << ".y * f" << j << ".y;";
        for (auto &lc : kv.second) o << " X" << lc.first << " += " << lit(lc.second, f32) << " * q;";
        o << " }\n";
      }
      for (int i = 0; i < n_lm; ++i) o << "        X" << i << " *= cc;\n";
      if (with_x)
        for (int i = 0; i < n_lm; ++i) {
          o << "        { real2 xv; xv.x = X" << i << "; xv.y = (real)0; xout[" << i << "LL * xslot + mo] = xv; }\n";
        }
    }
    o << "        if (bin >= 0) {\n";
    o << "          const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;\n";
    o << "          const double r2 = (double)n2; const double ir = bym_rsqrt(r2);\n";
    o << "          const double ux = nx * ir, uy = ny * ir, uz = nz * ir; const double zm = 1.0;\n";
    {
      std::ostringstream yy;
      emit_ylm(yy, L, false, "yk", "ux", "uy", "uz", "zm", f32);
      std::string s = yy.str();
      std::istringstream is(s);
      std::string line;
      while (std::getline(is, line)) o << "        " << line << "\n";
    }
    for (int l = 0; l <= L; l += 2) {
      o << "          { double T = 0.0;";
      for (int mu = -l; mu <= l; ++mu) o << " T += yk" << ylm_index(l, mu) << " * (double)X" << even_lm_index(l, mu) << ";";
      o << " v[" << l / 2 << "] = w * T; }\n";
    }
    o << "        }\n      }\n    }\n";
    o << "    bym_bin_flush<" << NL << ", double>(bin, v, s, nbins * " << NL << ");\n  }\n  bym_bins_out(s, gsum, nbins * " << NL << ");\n}\n";
  };
  emit_kcontract("kcontract", false);
  if (key.los == 2) emit_kcontract("kcontract_x", true);

  // ------------------------------------------------------------------ midpoint combine
  if (midpoint) emit_mid_combine(o, "mid_combine", key, midpoint_terms(key.ell_max, key.K, even), 0, nf, false);

  // ------------------------------------------------------------------ xi on the lag cube
  const int jlag = emit_xi_lag(o, "xi_lag", key, 0, nf);

  if (meta) {
    meta->key = key;
    meta->fields = F.list;
    meta->n_lm = n_lm;
    meta->n_ell = NL;
    meta->jmax_lag = jlag;
  }
  return o.str();
}

std::string generate_chunk_source(const JitKey &key, int max_fields, ChunkSet *meta) {
  const bool f32 = key.prec == 32;
  const char *real = f32 ? "float" : "double";
  const Fields F = field_set(key);
  const int nf = (int)F.list.size();
  const bool even = key.los == 3;
  std::vector<std::pair<int, int>> ranges;
  for (int f0 = 0; f0 < nf; f0 += max_fields) ranges.push_back({f0, std::min(nf, f0 + max_fields)});
  std::ostringstream o;
  o << "typedef " << real << " real;\ntypedef " << real << "2 real2;\n";
  o << kPrelude;
  if (key.los == 2) {   // bisector: field blocks and one contraction per block pair a <= b
    const int nb = (int)ranges.size();
    for (int a = 0; a < nb; ++a) {
      emit_gen_fields(o, ("gen_fields_c" + std::to_string(a)).c_str(), F.list, ranges[a].first, ranges[a].second,
                      key.prec == 32);
      for (int b = a; b < nb; ++b)
        emit_kcontract_pair(o, ("kcontract_p" + std::to_string(a) + "_" + std::to_string(b)).c_str(), key,
                            ranges[a].first, ranges[a].second, ranges[b].first, ranges[b].second);
    }
    if (meta) meta->ranges = ranges;
    return o.str();
  }
  const auto terms = midpoint_terms(key.ell_max, key.K, even);
  for (size_t q = 0; q < ranges.size(); ++q) {
    const std::string sfx = "_c" + std::to_string(q);
    emit_gen_fields(o, ("gen_fields" + sfx).c_str(), F.list, ranges[q].first, ranges[q].second, key.prec == 32);
    emit_mid_combine(o, ("mid_combine" + sfx).c_str(), key, terms, ranges[q].first, ranges[q].second, q > 0);
    emit_xi_lag(o, ("xi_lag" + sfx).c_str(), key, ranges[q].first, ranges[q].second);
  }
  if (meta) meta->ranges = ranges;
  return o.str();
}

std::string generate_cross_source(const JitKey &key) {
  const bool f32 = key.prec == 32;
  const char *real = f32 ? "float" : "double";
  const int nf = (int)field_set(key).list.size();
  std::ostringstream o;
  o << "typedef " << real << " real;\ntypedef " << real << "2 real2;\n";
  o << kPrelude;
  emit_kcontract_pair(o, "kcontract_cross", key, 0, nf, 0, nf, true);
  return o.str();
}

// ---------------------------------------------------------------------------
// Odd multipoles (l = 1, 3, .., ell_max, ell_max odd) of cross spectra, in a module of
// their own.  Outputs are indexed by odd_lm_index (fields / X slots) and (l - 1) / 2
// (shell sums).  A P_l of odd l is the imaginary part of the shell mean of
// sum_nu Y_{l nu}(k) X_{l nu}(k); xi_l is real.
// ---------------------------------------------------------------------------
namespace {

std::vector<FieldInfo> odd_field_list(const JitKey &key) {
  std::vector<FieldInfo> list;
  if (key.los == 1) {                       // midpoint: g^alpha_{J nu} with J - alpha odd
    for (auto &g : midpoint_gfields_odd(key.ell_max, key.K)) list.push_back({g.alpha, g.J, g.nu});
  } else if (key.los == 0) {                // Yamamoto: Y_{l nu} delta, odd l
    for (int l = 1; l <= key.ell_max; l += 2)
      for (int nu = -l; nu <= l; ++nu) list.push_back({0, l, nu});
  } else {                                  // bisector: Y_{J nu} delta, J <= ell_max + floor(K/2)
    const int Jmax = key.ell_max + key.K / 2;
    for (int J = 0; J <= Jmax; ++J)
      for (int nu = -J; nu <= J; ++nu) list.push_back({0, J, nu});
  }
  return list;
}

void emit_k_head(std::ostream &o, int NLo) {
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * " << NLo << ");\n  const int H = N / 2 + 1;\n";
  emit_bin_loop_head(o, "(long long)N * N * H");
  o << "    int bin = -1; double v[" << NLo << "] = {";
  for (int l = 0; l < NLo; ++l) o << (l ? ", " : "") << "0.0";
  o << "};\n";
  o << "    if (m < total) {\n";
  o << "      const int iz = (int)(m % H); const long long row = m / H, mo = row * (H + 1) + iz;\n";
  o << "      const int ix = (int)(row / N), iy = (int)(row % N);\n";
  o << "      const int nx = bym_lab(ix, N), ny = bym_lab(iy, N), nz = (iz == N / 2) ? -N / 2 : iz;\n";
  o << "      const int n2 = nx * nx + ny * ny + nz * nz;\n";
  o << "      bin = lut[n2];\n";
}

// shell sums of the odd l from X<odd_lm>: v[(l - 1) / 2] = w sum_nu Y_{l nu}(k) X_{l nu}
void emit_k_tail(std::ostream &o, int L, bool f32, int NLo) {
  o << "        if (bin >= 0) {\n";
  o << "          const double w = (iz == 0 || iz == N / 2) ? 1.0 : 2.0;\n";
  o << "          const double r2 = (double)n2; const double ir = bym_rsqrt(r2);\n";
  o << "          const double ux = nx * ir, uy = ny * ir, uz = nz * ir; const double zm = 1.0;\n";
  {
    std::ostringstream yy;
    emit_ylm(yy, L, false, "yk", "ux", "uy", "uz", "zm", f32);
    std::istringstream is(yy.str());
    std::string line;
    while (std::getline(is, line)) o << "        " << line << "\n";
  }
  for (int l = 1; l <= L; l += 2) {
    o << "          { double T = 0.0;";
    for (int mu = -l; mu <= l; ++mu) o << " T += yk" << ylm_index(l, mu) << " * (double)X" << odd_lm_index(l, mu) << ";";
    o << " v[" << (l - 1) / 2 << "] = w * T; }\n";
  }
  o << "        }\n      }\n    }\n";
  o << "    bym_bin_flush<" << NLo << ", double>(bin, v, s, nbins * " << NLo << ");\n  }\n  bym_bins_out(s, gsum, nbins * " << NLo << ");\n}\n";
}

}  // namespace

std::string generate_odd_source(const JitKey &key, OddSet *meta) {
  if (key.ell_max < 1 || key.ell_max % 2 == 0 || key.los < 0 || key.los > 2)
    throw std::runtime_error("odd multipoles: odd ell_max, Yamamoto, midpoint or bisector");
  const bool f32 = key.prec == 32;
  const char *real = f32 ? "float" : "double";
  const int L = key.ell_max, NLo = (L + 1) / 2, n_lm = n_odd_lm(L);
  const auto list = odd_field_list(key);
  const int nf = (int)list.size();
  std::ostringstream o;
  o << "typedef " << real << " real;\ntypedef " << real << "2 real2;\n";
  o << kPrelude;
  emit_gen_fields(o, "gen_fields_odd", list, 0, nf, key.prec == 32);

  if (key.los == 1) {
    // midpoint: H_{l nu}(Delta) = sum phi Y_{J1}(Delta) t^alpha g^alpha_{J2}(Delta) over the odd-l g fields
    // (mid_combine_odd), then X_{l nu} = Im F[H_{l nu}](k) (kcontract_mid_odd)
    emit_mid_combine(o, "mid_combine_odd", key, midpoint_terms_odd(key.ell_max, key.K), 0, nf, false, n_lm);
    o << "extern \"C\" __global__ void __launch_bounds__(256) kcontract_mid_odd(const real2* __restrict__ F,"
         " long long cslot, int N, const int* __restrict__ lut, int nbins, double* __restrict__ gsum) {\n";
    emit_k_head(o, NLo);
    o << "      if (bin >= 0) {\n";
    for (int i = 0; i < n_lm; ++i) o << "        const real X" << i << " = F[" << i << "LL * cslot + mo].y;\n";
    emit_k_tail(o, L, f32, NLo);
  } else if (key.los == 0) {
    // Yamamoto: X_{l nu} = sgn Im(F_{l nu}(k) conj D(k)) W^-2; two launches (F^B with D_A, sgn 1;
    // F^A with D_B, sgn -1) add [Q^AB - Q^BA], halved on the host
    o << "extern \"C\" __global__ void __launch_bounds__(256) kcontract_odd(const real2* __restrict__ F, long long cslot,"
         " const real2* __restrict__ D, int N, const int* __restrict__ lut, int nbins, double* __restrict__ gsum,"
         " const real* __restrict__ invw, real sgn) {\n";
    emit_k_head(o, NLo);
    o << "      if (bin >= 0) {\n";
    o << "        real cc = sgn;\n";
    o << "        if (invw) { const real wv = invw[ix] * invw[iy] * invw[iz]; cc = sgn * wv * wv; }\n";
    o << "        const real2 d = D[mo];\n";
    for (int i = 0; i < nf; ++i)
      o << "        real X" << odd_lm_index(list[i].J, list[i].nu) << "; { const real2 f = F[" << i
        << "LL * cslot + mo]; X" << odd_lm_index(list[i].J, list[i].nu) << " = (f.y * d.x - f.x * d.y) * cc; }\n";
    emit_k_tail(o, L, f32, NLo);
  } else {
    // bisector: X_{l nu}(k) = sum over ordered field pairs c_ij Im(conj F^A_i F^B_j) W^-2, the part of
    // the bilinear sum of eq. bisector-pk-fft that is odd in k; xout (for xi) gets i X
    o << "extern \"C\" __global__ void __launch_bounds__(256) kcontract_cross_odd(const real2* __restrict__ FA,"
         " const real2* __restrict__ FB, long long cslot, int N, const int* __restrict__ lut, int nbins,"
         " double* __restrict__ gsum, real2* __restrict__ xout, long long xslot, const real* __restrict__ invw) {\n";
    emit_k_head(o, NLo);
    o << "      if (xout || bin >= 0) {\n";
    o << "        real cc = (real)1;\n";
    o << "        if (invw) { cc = invw[ix] * invw[iy] * invw[iz]; cc = cc * cc; }\n";
    for (int i = 0; i < n_lm; ++i) o << "        real X" << i << " = (real)0;\n";
    std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> by_pair;
    for (auto &t : bisector_terms_odd(key.ell_max, key.K)) {
      if (t.i == t.j) {
        by_pair[{t.i, t.j}].push_back({t.lm, t.c});
      } else {
        by_pair[{t.i, t.j}].push_back({t.lm, 0.5 * t.c});
        by_pair[{t.j, t.i}].push_back({t.lm, 0.5 * t.c});
      }
    }
    std::set<int> ub;
    for (auto &kv : by_pair) ub.insert(kv.first.second);
    for (int j : ub) o << "        const real2 b" << j << " = FB[" << j << "LL * cslot + mo];\n";
    int cur = -1;
    for (auto &kv : by_pair) {
      const int i = kv.first.first, j = kv.first.second;
      if (i != cur) {
        if (cur >= 0) o << "        }\n";
        o << "        { const real2 a" << i << " = FA[" << i << "LL * cslot + mo];\n";
        cur = i;
      }
      o << "        { const real q = a" << i << ".x * b" << j << ".y - a" << i << ".y * b" << j << ".x;";
      for (auto &lc : kv.second) o << " X" << lc.first << " += " << lit(lc.second, f32) << " * q;";
      o << " }\n";
    }
    if (cur >= 0) o << "        }\n";
    for (int i = 0; i < n_lm; ++i) o << "        X" << i << " *= cc;\n";
    o << "        if (xout) {\n";
    for (int i = 0; i < n_lm; ++i)
      o << "          { real2 xv; xv.x = (real)0; xv.y = X" << i << "; xout[" << i << "LL * xslot + mo] = xv; }\n";
    o << "        }\n";
    emit_k_tail(o, L, f32, NLo);
  }

  // xi on the lag cube: T_l(Delta) = sum_nu Y_{l nu}(Delta) Z_{l nu}(Delta), Z in odd_lm order; midpoint:
  // T_l(Delta) = sum f t^alpha sum_nu Y_{J nu}(Delta) g^alpha_{J nu}(Delta) over the odd-l g fields
  std::vector<XiTerm> xterms;
  int jlag = L;
  if (key.los == 1) {
    xterms = midpoint_xi_terms_odd(key.ell_max, key.K);
    for (auto &x : xterms) jlag = std::max(jlag, x.J);
  }
  o << "extern \"C\" __global__ void __launch_bounds__(256) xi_lag_odd(const real* __restrict__ Z, long long slot,"
       " int N, int jm, int full, const int* __restrict__ lut, int nbins, double* __restrict__ gsum,"
       " double zscale, double tscale) {\n";
  o << "  extern __shared__ double s[];\n  bym_bins_init(s, nbins * " << NLo << ");\n";
  o << "  const int Lc = full ? N : 2 * jm + 1;\n";
  emit_bin_loop_head(o, "(long long)Lc * Lc * Lc");
  o << "    int bin = -1; double v[" << NLo << "] = {";
  for (int l = 0; l < NLo; ++l) o << (l ? ", " : "") << "0.0";
  o << "};\n";
  o << "    if (m < total) {\n";
  o << "      const int a = (int)(m % Lc); const long long t = m / Lc;\n";
  o << "      const int b = (int)(t % Lc); const int c = (int)(t / Lc);\n";
  o << "      const int jx = full ? bym_lab(c, N) : c - jm, jy = full ? bym_lab(b, N) : b - jm,"
       " jz = full ? bym_lab(a, N) : a - jm;\n";
  o << "      const int j2 = jx * jx + jy * jy + jz * jz;\n";
  o << "      bin = lut[j2];\n";
  o << "      if (bin >= 0) {\n";
  o << "        const int ix = jx < 0 ? jx + N : jx, iy = jy < 0 ? jy + N : jy, iz = jz < 0 ? jz + N : jz;\n";
  o << "        const long long off = ((long long)ix * N + iy) * (N + 4) + iz;\n";
  o << "        const double rr = sqrt((double)j2); const double ir = 1.0 / rr;\n";
  o << "        const double ux = jx * ir, uy = jy * ir, uz = jz * ir, zm = 1.0;\n";
  {
    std::ostringstream yy;
    emit_ylm(yy, jlag, false, "yl", "ux", "uy", "uz", "zm");
    std::istringstream is(yy.str());
    std::string line;
    while (std::getline(is, line)) o << "      " << line << "\n";
  }
  if (key.los == 1) {
    o << "        const double t1 = rr * tscale;\n";
    for (int a2 = 2; a2 <= key.K; ++a2) o << "        const double t" << a2 << " = t" << a2 - 1 << " * t1;\n";
    for (int l = 1; l <= L; l += 2) {
      o << "        { double T = 0.0;\n";
      for (auto &x : xterms) {
        if (x.l != l) continue;
        o << "          { double S = 0.0;";
        for (int nu = -x.J; nu <= x.J; ++nu)
          o << " S += yl" << ylm_index(x.J, nu) << " * (double)Z["
            << midpoint_gfield_index_odd(key.ell_max, x.alpha, x.J, nu) << "LL * slot + off];";
        o << " T += " << lit(x.f, false);
        if (x.alpha > 0) o << " * t" << x.alpha;
        o << " * S; }\n";
      }
      o << "          v[" << (l - 1) / 2 << "] = T * zscale; }\n";
    }
  } else {
    for (int l = 1; l <= L; l += 2) {
      o << "        { double T = 0.0;";
      for (int mu = -l; mu <= l; ++mu)
        o << " T += yl" << ylm_index(l, mu) << " * (double)Z[" << odd_lm_index(l, mu) << "LL * slot + off];";
      o << " v[" << (l - 1) / 2 << "] = T * zscale; }\n";
    }
  }
  o << "      }\n    }\n";
  o << "    bym_bin_flush<" << NLo << ", double>(bin, v, s, nbins * " << NLo << ");\n  }\n  bym_bins_out(s, gsum, nbins * " << NLo << ");\n}\n";

  if (meta) {
    meta->fields = list;
    meta->n_lm = n_lm;
    meta->n_ell = NLo;
  }
  return o.str();
}

bool compile_cubin(const std::string &src, std::vector<char> &cubin, std::string &log) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "bym_generated.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    log = "nvrtcCreateProgram failed";
    return false;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "-lineinfo",
                        "-diag-suppress=177,550"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, 5, opts);
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  log.assign(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &log[0]);
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t cn = 0;
  nvrtcGetCUBINSize(prog, &cn);
  cubin.resize(cn);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return true;
}

std::shared_ptr<KernelSet> get_kernels(const JitKey &key, std::string &err) {
  static std::mutex mu;
  static std::map<JitKey, std::shared_ptr<KernelSet>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  auto ks = std::make_shared<KernelSet>();
  std::string src;
  try {
    src = generate_source(key, ks.get());
  } catch (const std::exception &e) {
    err = std::string("kernel generation failed: ") + e.what();
    return nullptr;
  }
  std::vector<char> cubin;
  std::string log;
  if (!compile_cubin(src, cubin, log)) {
    err = "NVRTC compile failed: " + log.substr(0, 2000);
    return nullptr;
  }
  if (cudaLibraryLoadData(&ks->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(cudaGetLastError());
    return nullptr;
  }
  auto get = [&](const char *name, cudaKernel_t *k) {
    if (cudaLibraryGetKernel(k, ks->lib, name) != cudaSuccess) {
      cudaGetLastError();
      *k = nullptr;
    }
  };
  get("gen_fields", &ks->gen_fields);
  get("kgeom", &ks->kgeom);
  get("rgeom", &ks->rgeom);
  get("kcontract", &ks->kcontract);
  get("kcontract_x", &ks->kcontract_x);
  get("mid_combine", &ks->mid_combine);
  get("xi_lag", &ks->xi_lag);
  if (!ks->gen_fields || !ks->kgeom || !ks->rgeom || !ks->kcontract || !ks->xi_lag) {
    err = "generated module is missing a kernel";
    return nullptr;
  }
  cache[key] = ks;
  return ks;
}

cudaKernel_t get_cross_kernel(const JitKey &key, std::string &err) {
  static std::mutex mu;
  static std::map<JitKey, cudaKernel_t> cache;
  if (key.los != 2) {
    err = "the two-set contraction belongs to the bisector";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::string src;
  try {
    src = generate_cross_source(key);
  } catch (const std::exception &e) {
    err = std::string("kernel generation failed: ") + e.what();
    return nullptr;
  }
  std::vector<char> cubin;
  std::string log;
  if (!compile_cubin(src, cubin, log)) {
    err = "NVRTC compile failed: " + log.substr(0, 2000);
    return nullptr;
  }
  cudaLibrary_t lib = nullptr;
  cudaKernel_t k = nullptr;
  if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&k, lib, "kcontract_cross") != cudaSuccess) {
    err = std::string("loading the cross contraction: ") + cudaGetErrorString(cudaGetLastError());
    return nullptr;
  }
  cache[key] = k;   // the library stays loaded for the life of the process, as the other modules do
  return k;
}

std::shared_ptr<OddSet> get_odd_kernels(const JitKey &key, std::string &err) {
  static std::mutex mu;
  static std::map<JitKey, std::shared_ptr<OddSet>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  auto os = std::make_shared<OddSet>();
  std::string src;
  try {
    src = generate_odd_source(key, os.get());
  } catch (const std::exception &e) {
    err = std::string("kernel generation failed: ") + e.what();
    return nullptr;
  }
  std::vector<char> cubin;
  std::string log;
  if (!compile_cubin(src, cubin, log)) {
    err = "NVRTC compile failed: " + log.substr(0, 2000);
    return nullptr;
  }
  if (cudaLibraryLoadData(&os->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(cudaGetLastError());
    return nullptr;
  }
  const char *kc = key.los == 0 ? "kcontract_odd" : key.los == 1 ? "kcontract_mid_odd" : "kcontract_cross_odd";
  if (cudaLibraryGetKernel(&os->gen_fields, os->lib, "gen_fields_odd") != cudaSuccess ||
      cudaLibraryGetKernel(&os->kcontract, os->lib, kc) != cudaSuccess ||
      cudaLibraryGetKernel(&os->xi_lag, os->lib, "xi_lag_odd") != cudaSuccess ||
      (key.los == 1 && cudaLibraryGetKernel(&os->mid_combine, os->lib, "mid_combine_odd") != cudaSuccess)) {
    cudaGetLastError();
    err = "generated odd-multipole module is missing a kernel";
    return nullptr;
  }
  cache[key] = os;
  return os;
}

std::shared_ptr<ChunkSet> get_chunk_kernels(const JitKey &key, int max_fields, std::string &err) {
  static std::mutex mu;
  static std::map<std::pair<JitKey, int>, std::shared_ptr<ChunkSet>> cache;
  if (key.los == 0 || max_fields < 1) {
    err = "field ranges apply to the midpoint forms and the bisector";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({key, max_fields});
  if (it != cache.end()) return it->second;
  auto cs = std::make_shared<ChunkSet>();
  std::string src;
  try {
    src = generate_chunk_source(key, max_fields, cs.get());
  } catch (const std::exception &e) {
    err = std::string("kernel generation failed: ") + e.what();
    return nullptr;
  }
  std::vector<char> cubin;
  std::string log;
  if (!compile_cubin(src, cubin, log)) {
    err = "NVRTC compile failed: " + log.substr(0, 2000);
    return nullptr;
  }
  if (cudaLibraryLoadData(&cs->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(cudaGetLastError());
    return nullptr;
  }
  if (key.los == 2) {
    const int nb = (int)cs->ranges.size();
    cs->pair.assign((size_t)nb * nb, nullptr);
    for (int a = 0; a < nb; ++a) {
      std::vector<std::string> names = {"gen_fields_c" + std::to_string(a)};
      for (int b = a; b < nb; ++b) names.push_back("kcontract_p" + std::to_string(a) + "_" + std::to_string(b));
      for (size_t n = 0; n < names.size(); ++n) {
        cudaKernel_t k = nullptr;
        if (cudaLibraryGetKernel(&k, cs->lib, names[n].c_str()) != cudaSuccess) {
          cudaGetLastError();
          err = "generated block module is missing " + names[n];
          return nullptr;
        }
        if (n == 0)
          cs->gen.push_back(k);
        else
          cs->pair[(size_t)a * nb + a + (n - 1)] = k;
      }
    }
    cache[{key, max_fields}] = cs;
    return cs;
  }
  for (size_t q = 0; q < cs->ranges.size(); ++q) {
    const std::string sfx = "_c" + std::to_string(q);
    cudaKernel_t k[3] = {nullptr, nullptr, nullptr};
    const std::string names[3] = {"gen_fields" + sfx, "mid_combine" + sfx, "xi_lag" + sfx};
    for (int i = 0; i < 3; ++i)
      if (cudaLibraryGetKernel(&k[i], cs->lib, names[i].c_str()) != cudaSuccess) {
        cudaGetLastError();
        err = "generated chunk module is missing " + names[i];
        return nullptr;
      }
    cs->gen.push_back(k[0]);
    cs->comb.push_back(k[1]);
    cs->xi.push_back(k[2]);
  }
  cache[{key, max_fields}] = cs;
  return cs;
}

}  // namespace bym
