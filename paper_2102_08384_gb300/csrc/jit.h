// Runtime-specialised kernels: for each (LOS, ell_max, order, precision) the
// generator writes straight-line CUDA C++ (unrolled real-harmonic recurrences,
// sparse couplings as immediates) and compiles it with NVRTC for sm_103a.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <utility>
#include <string>
#include <vector>

namespace bym {

struct JitKey {
  int los, ell_max, K, prec;
  bool operator<(const JitKey &o) const {
    if (los != o.los) return los < o.los;
    if (ell_max != o.ell_max) return ell_max < o.ell_max;
    if (K != o.K) return K < o.K;
    return prec < o.prec;
  }
};

struct FieldInfo { int alpha, J, nu; };

struct KernelSet {
  JitKey key;
  std::vector<FieldInfo> fields;   // fields written by gen_fields, in slot order
  int n_lm = 0;                    // number of (ell, mu) outputs, even ell <= ell_max
  int n_ell = 0;                   // ell = 0, 2, .., ell_max
  int jmax_lag = 0;                // harmonic degree needed on the lag grid by xi_lag
  cudaLibrary_t lib = nullptr;
  cudaKernel_t gen_fields = nullptr, kgeom = nullptr, rgeom = nullptr;
  cudaKernel_t kcontract = nullptr, kcontract_x = nullptr, mid_combine = nullptr, xi_lag = nullptr;
};

// Field sets under a memory bound.  Midpoint forms: the g fields in ranges of at
// most max_fields, each with its own gen_fields / mid_combine (accumulating into H
// after the first range) / xi_lag (adding its share of the shell sums).  Bisector:
// the fields in blocks of at most max_fields, gen_fields per block and one
// contraction per block pair a <= b (pair[a * nblocks + b]).
struct ChunkSet {
  std::vector<std::pair<int, int>> ranges;   // field ranges [f0, f1) in slot order
  cudaLibrary_t lib = nullptr;
  std::vector<cudaKernel_t> gen, comb, xi;   // one of each per range (bisector: gen only)
  std::vector<cudaKernel_t> pair;            // bisector block-pair contractions
};

// Source text for a configuration (exposed for build checks).
std::string generate_source(const JitKey &key, KernelSet *meta);

std::string generate_chunk_source(const JitKey &key, int max_fields, ChunkSet *meta);

// Bisector cross spectra of two tracers: kcontract_cross(FA, FB, ...) with the arguments of
// the block-pair contraction, FA / FB every field F[Y_J^M delta] of tracer A / B, summing
// X_{lm}(k) = sum c_ij Re(conj F^A_i F^B_j) over ordered pairs (the Hermitian part of eq.
// bisector-pk-fft with delta_A at r_1, delta_B at r_2).
std::string generate_cross_source(const JitKey &key);
cudaKernel_t get_cross_kernel(const JitKey &key, std::string &err);

// Odd multipoles l = 1, 3, .., ell_max (key.ell_max odd) of cross spectra, Yamamoto (los 0),
// midpoint (los 1, all-parity series) or bisector (los 2): gen_fields_odd (Yamamoto: Y_{l nu} delta
// for odd l; midpoint: the g fields with J - alpha odd; bisector: Y_{J nu} delta, J <= ell_max +
// floor(K/2)), the contraction (Yamamoto kcontract_odd(F, cslot, D, N, lut, nbins, gsum, invw, sgn):
// sgn Im(F conj D) W^-2; midpoint mid_combine_odd and kcontract_mid_odd(F, cslot, N, lut, nbins,
// gsum): Im F[H]; bisector kcontract_cross_odd with the arguments of kcontract_cross: sum c_ij
// Im(conj F^A_i F^B_j) W^-2, xout = i X) and xi_lag_odd(Z, slot, N, jm, full, lut, nbins, gsum,
// zscale, tscale).  Shell sums [bin][(l - 1) / 2]; X, H and Z slots in odd_lm_index order (midpoint
// Z: the g fields in midpoint_gfield_index_odd order).
struct OddSet {
  std::vector<FieldInfo> fields;
  int n_lm = 0, n_ell = 0;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t gen_fields = nullptr, kcontract = nullptr, xi_lag = nullptr;
  cudaKernel_t mid_combine = nullptr;   // midpoint: mid_combine_odd(G, slot, Hout, N, tscale)
};
std::string generate_odd_source(const JitKey &key, OddSet *meta);
std::shared_ptr<OddSet> get_odd_kernels(const JitKey &key, std::string &err);

// Compile to a cubin for sm_103a; returns false and fills log on failure.
bool compile_cubin(const std::string &src, std::vector<char> &cubin, std::string &log);

// Process-wide cache: generate, compile, load.  Thread-safe.
std::shared_ptr<KernelSet> get_kernels(const JitKey &key, std::string &err);
std::shared_ptr<ChunkSet> get_chunk_kernels(const JitKey &key, int max_fields, std::string &err);

}  // namespace bym
