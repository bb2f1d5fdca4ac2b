// Native FP32 3D FFTs of 512^3 meshes (fft512.cu), in the padded in-place slot layout.
#pragma once
#include <cuda_runtime.h>

namespace bym {

bool native_fft_supported(int n_mesh, int precision);
cudaError_t native_fft_prepare();  // per device: twiddle table, shared-memory attributes
// forward R2C / inverse C2R (unnormalised) of slots [first, first + count); cluster = CTAs per
// thread-block cluster in the plane pass, 8 or 16 (16 is a non-portable cluster size)
cudaError_t native_fft_forward(float *slots, long long slot_reals, int first, int count, int cluster,
                               cudaStream_t st);
cudaError_t native_fft_inverse(float *slots, long long slot_reals, int first, int count, int cluster,
                               cudaStream_t st);
// for each slot f: real field -> forward -> * conj(D) scale[f] W(k)^-2 -> inverse, in place
// (D: the half-spectrum of delta; invw: per-axis 1/W or null)
cudaError_t native_fft_convolve(float *slots, long long slot_reals, int first, int count, const float *D,
                                const double *scale, const float *invw, int cluster, cudaStream_t st);

// whether an x pass on device dev gave up waiting for a tile copy (that kernel returned early
// and its output is incomplete); read from mapped host memory after the stream has synchronised;
// the flag stays set for the device's lifetime
bool native_fft_fault(int dev);

// The library's own (y, z) plane transforms of slots [first, first + count), in two passes:
// the z pass (R2C / C2R along z of blocks of 32 whole rows, moved by bulk copies) and the y pass
// (C2C along y of tiles of 16 kz columns, moved by TMA like the x pass's).  A forward transform
// runs the z pass then the y pass, an inverse one the y pass then the z pass.  Both cover the x
// planes [xlo, xhi); the forward z pass transforms the rows y in [ylo, yhi) of them only and the
// forward y pass reads only those rows (the others hold zeros, whose transforms are zeros in the
// same bytes); mode-1 (inverse) calls read every row.  xlo, xhi, ylo, yhi are multiples of 32.
cudaError_t native_fft_zpass(int inverse, float *slots, long long slot_reals, int first, int count, cudaStream_t st,
                             int xlo = 0, int xhi = 512, int ylo = 0, int yhi = 512);
cudaError_t native_fft_ypass(int inverse, float *slots, long long slot_reals, int first, int count, cudaStream_t st,
                             int xlo = 0, int xhi = 512, int ylo = 0, int yhi = 512);

// the x pass alone (C2C along x of half spectra) for slots [first, first + count):
// mode 0 forward, 1 inverse, 2 forward -> * conj(D) scale[f] W(k)^-2 -> inverse.  Modes 0 and 2
// read the input rows x in [xlo, xhi) only and take the others as zero (planes that hold no
// painted value); the output covers every x.  xlo and xhi are multiples of 32; the slots and D
// start on 16-byte boundaries.
cudaError_t native_fft_xpass(int mode, float *slots, long long slot_reals, int first, int count, const float *D,
                             const double *scale, const float *invw, cudaStream_t st, int xlo = 0, int xhi = 512);

}  // namespace bym
