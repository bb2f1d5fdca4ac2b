// Native FP32 3D FFTs of 512^3 meshes (fft512.cu), in the padded in-place slot layout.
#pragma once
#include <cuda_runtime.h>

namespace bym {

bool native_fft_supported(int n_mesh, int precision);
cudaError_t native_fft_prepare();  // per device: twiddle table, shared-memory attributes
// forward R2C / inverse C2R (unnormalised) of slots [first, first + count)
cudaError_t native_fft_forward(float *slots, long long slot_reals, int first, int count, cudaStream_t st);
cudaError_t native_fft_inverse(float *slots, long long slot_reals, int first, int count, cudaStream_t st);
// for each slot f: real field -> forward -> * conj(D) scale[f] W(k)^-2 -> inverse, in place
// (D: the half-spectrum of delta; invw: per-axis 1/W or null)
cudaError_t native_fft_convolve(float *slots, long long slot_reals, int first, int count, const float *D,
                                const double *scale, const float *invw, cudaStream_t st);

}  // namespace bym
