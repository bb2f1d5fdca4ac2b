// Launchers of the ahead-of-time kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>

namespace bym {

void launch_norm_reduce(const float4 *p, const float *nbar, long long n, int which, const double lo[3], double inv_h,
                        int N, double *stats, int nsm, cudaStream_t st);

template <typename T>
void launch_paint(const float4 *p, long long n, int is_ran, const double *stats, T *delta, int N, const double lo[3],
                  double inv_h, int assign, int nsm, cudaStream_t st);

template <typename T, typename T2>
void launch_spec_mul(T2 *F, long long cslot, int nf, const T2 *D, int N, const double *scale, const T *invw, int nsm,
                     cudaStream_t st);

}  // namespace bym
