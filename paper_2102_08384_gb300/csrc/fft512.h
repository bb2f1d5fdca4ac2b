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

// the x pass alone (C2C along x of half spectra) for slots [first, first + count):
// mode 0 forward, 1 inverse, 2 forward -> * conj(D) scale[f] W(k)^-2 -> inverse.  Modes 0 and 2
// read the input rows x in [xlo, xhi) only and take the others as zero (planes that hold no
// painted value); the output covers every x.  xlo and xhi are multiples of 32; the slots and D
// start on 16-byte boundaries.
cudaError_t native_fft_xpass(int mode, float *slots, long long slot_reals, int first, int count, const float *D,
                             const double *scale, const float *invw, cudaStream_t st, int xlo = 0, int xhi = 512);

}  // namespace bym
