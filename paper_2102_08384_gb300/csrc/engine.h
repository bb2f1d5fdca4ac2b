// Internal interfaces of the request engine shared by engine.cu and serve.cpp.
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bym.h"

namespace bym {

struct Geom {
  int *lut = nullptr;           // device: bin of each |n|^2 (or -1)
  int nbins = 0;
  int jm = 0, full = 0;         // lag cube half-width (r bins only)
  std::vector<int64_t> count;   // modes / lag cells per bin (full grid)
  std::vector<double> mean;     // mean |k| or |Delta| per bin
  long long half_binned = 0;    // k bins: half-spectrum modes in some bin (the modes a contraction reads)
};

struct Request {
  const bym_catalog *gal, *ran;
  const bym_params *p;
  const bym_bins *kb, *rb;      // NULL: that statistic is not requested
  double *pk, *kmean;
  int64_t *nmodes;
  double *xi, *rmean;
  int64_t *ncells;
  double *alpha = nullptr;      // optional out: alpha_r = sum w_g / sum w_r of the request
  const bym_catalog *gal_b = nullptr, *ran_b = nullptr;   // second tracer of a cross spectrum (else NULL)
  bool odd = false;             // the odd multipoles of a cross spectrum (p->ell_max odd)
  bool full_planes = false;     // transform every x plane (as requests captured into graphs do)
};

struct Server;  // serving loop state (serve.cpp)

// Launch shapes chosen by bym_autotune for one (n_mesh, precision, LOS).
struct Tune {
  int per_sm_gen = 16;    // blocks per SM of gen_fields (grid-stride, 256 threads)
  int per_sm_comb = 16;   // mid_combine
  int per_sm_k = 4;       // kcontract / kcontract_x
  int per_sm_spec = 8;    // spec_mul
  int fft_batch = 8;      // transforms per cuFFT call
  int native = -1;        // FFT path: 0 cuFFT 3D, 1 cuFFT planes + library x pass, 2 cuFFT planes + cuFFT x,
                          // 8 / 16 library two-pass (CTAs per plane-pass cluster); -1 untuned: 1 where the
                          // library's kernels apply (512^3 FP32), else 0
};

struct ProfEntry {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0;
};
struct ProfPending {
  std::string name;
  cudaEvent_t a, b;
  double bytes;
};

}  // namespace bym

struct bym_ctx {
  int device = 0;
  size_t budget = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::mutex mu;                                               // one request at a time per context
  std::map<std::tuple<int, int, int, int>, cufftHandle> plans;  // (N, precision, inverse, batch)
  void *fft_work = nullptr;
  size_t fft_work_size = 0;
  std::map<std::string, bym::Geom> kgeo, rgeo;
  bym::Server *server = nullptr;
  std::set<std::string> graph_warm;  // request shapes bym_batch_graph has warmed on this context
  int field_chunk = 0;  // midpoint g fields per streamed range: 0 = only when the whole set does not fit
  int fft_mode = 2;  // 0 cuFFT, 1 library FFT kernels (8-CTA clusters), 2 as tuned, 3 library (16-CTA clusters)
  std::map<std::tuple<int, int, int>, bym::Tune> tune;         // (n_mesh, precision, los) -> launch shapes
  bool prof = false;                                           // kernel tracing (bym_profile_enable)
  std::map<std::string, bym::ProfEntry> prof_tab;
  std::vector<bym::ProfPending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
};

namespace bym {

int validate_params(bym_ctx *c, const bym_params *p);
int validate(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p, const bym_bins *kb,
             const bym_bins *rb);
// Device bytes one request holds.  chunk > 0: the midpoint g fields are streamed
// in ranges of at most chunk fields (two delta slots, one range, the H fields).
// cross: two tracers, each with its own delta and field set (n_gal, n_ran summed over both).
size_t footprint_bytes(const bym_params *p, int64_t n_gal, int64_t n_ran, bool want_pk, bool want_xi,
                       bool cats_on_device, int chunk = 0, bool cross = false);
int run_request(bym_ctx *c, const Request &rq, cudaStream_t st);
// device bytes still available to requests: free memory plus what the stream-ordered pool holds
// unused (it keeps freed memory between requests), less headroom
size_t device_available(bym_ctx *c, size_t headroom);
void shutdown_serving(bym_ctx *c);

}  // namespace bym
