// Launchers of the ahead-of-time kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>

namespace bym {

// Padded in-place layout of a mesh slot: N x N rows of N + kRowPad reals, or N / 2 + 2 complex
// values of which kz = 0..N/2 hold the half spectrum and the last is padding.  Four padding reals
// (not the two an in-place transform needs) put every row on a 16-byte boundary (2064 bytes at
// N = 512 in FP32), which lets the tensor memory accelerator move tiles along y.
constexpr int kRowPad = 4;

// Catalog sums into stats (see bym_norm_reduce), deterministic: per-block partials in part
// (norm_scratch_bytes(nsm) bytes of device scratch), added up in block order.
size_t norm_scratch_bytes(int nsm);
// precision 32: the in-box test runs as the FP32 painter's (float pairs), 64: in FP64.
void launch_norm_reduce(const float4 *p, const float *nbar, long long n, int which, const double lo[3], double inv_h,
                        int N, double *stats, double *part, int nsm, cudaStream_t st, int precision);

// Device scratch of launch_paint for a mesh of N^3 and n_objects galaxies plus randoms.
size_t paint_scratch_bytes(int N, long long n_objects);

// delta = paint(gal, +w) + paint(ran, -alpha_r w), alpha_r = stats[0] / stats[1]; every cell of the
// padded slot is written (no zero-fill needed), deterministically.  stats[6], stats[7] hold
// the largest |w| of the galaxies and of the randoms (the scale of the fixed-point sums).  shift (cells): paint
// onto the nodes box_lo + (i + shift) h (interlacing uses 1/2).  ng + nr < 2^32.
template <typename T>
cudaError_t launch_paint(const float4 *gal, long long ng, const float4 *ran, long long nr, const double *stats,
                         T *delta, int N, const double lo[3], double inv_h, int assign, void *scratch, int nsm,
                         cudaStream_t st, double shift = 0.0);

template <typename T, typename T2>
void launch_spec_mul(T2 *F, long long cslot, int nf, const T2 *D, int N, const double *scale, const T *invw, int nsm,
                     cudaStream_t st);

// two tracers: FA_f <- [sa FA_f conj(DB) + FB_f conj(DA)] scale_f W^-2 / 2 (half-spectrum slots)
template <typename T, typename T2>
void launch_spec_mul_cross(T2 *FA, const T2 *FB, long long cslot, int nf, const T2 *DA, const T2 *DB, int N,
                           const double *scale, const T *invw, int nsm, cudaStream_t st, double sa = 1.0);

// the x planes of a padded real slot holding non-zero values: range[0] = min(range[0], x),
// range[1] = max(range[1], x) over them, and range[2], range[3] likewise for the rows y that hold
// one in any plane (set range to {N, -1, N, -1} before the first call)
template <typename T>
void launch_plane_range(const T *slot, int N, int *range, cudaStream_t st);

// F_f <- (F_f + P G_f) / 2, P(k) = ph[n_x] ph[n_y] ph[n_z] (half-spectrum slots)
template <typename T, typename T2>
void launch_interlace(T2 *F, const T2 *G, long long cslot, int nf, int N, const T2 *ph, int nsm, cudaStream_t st);

}  // namespace bym
