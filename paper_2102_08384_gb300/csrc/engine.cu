// Request engine and C ABI: validation, device buffers, cuFFT plans, shell
// geometry caches and the launch sequence of each estimator (include/bym.h).
//
// Launch sequence of one request (all on the caller's stream):
//   norm_reduce (gal, ran) -> paint (gal, ran) -> gen_fields -> batched R2C
//   Yamamoto : kcontract                      | spec_mul -> C2R -> xi_lag
//   midpoint : spec_mul -> C2R -> [xi_lag] -> [mid_combine -> R2C(H) -> kcontract]
//   bisector : kcontract (or kcontract_x -> C2R(X) -> xi_lag)
// then one device-to-host copy of the FP64 shell sums.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "bym.h"
#include "coeff.h"
#include "engine.h"
#include "fft512.h"
#include "jit.h"
#include "kernels.cuh"

using namespace bym;

namespace {

int fail(bym_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

// Device allocations of one request, released in stream order.
struct DevBufs {
  cudaStream_t st;
  std::vector<void *> ptrs;
  explicit DevBufs(cudaStream_t s) : st(s) {}
  ~DevBufs() {
    for (void *p : ptrs) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

template <class... A>
cudaError_t launch(cudaKernel_t k, unsigned grid, unsigned block, size_t smem, cudaStream_t st, A... args) {
  void *argv[] = {(void *)&args...};
  return cudaLaunchKernel((const void *)k, dim3(grid), dim3(block), argv, smem, st);
}

#define TRY_RC(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

unsigned grid_of(long long work, int nsm, int per_sm) {
  long long g = (work + 255) / 256;
  const long long cap = (long long)nsm * per_sm;
  return (unsigned)std::max(1LL, std::min(g, cap));
}

// Dynamic shared memory of a shell-sum kernel over n sums: one accumulator per warp of a
// 256-thread block when that fits the default 48 KB (the sums then do not depend on the order
// in which blocks and warps finish), else one per block.
size_t sums_smem(int n) {
  const size_t per_warp = sizeof(double) * 8 * (size_t)n;
  return per_warp <= 48 * 1024 ? per_warp : sizeof(double) * (size_t)n;
}

// Doubles of a shell-sum buffer: the n sums, a ticket counter, and one total per block of the
// largest grid that adds into it (nsm * per_sm blocks at most, see grid_of).
size_t sums_doubles(int n, int nsm, int per_sm) { return (size_t)n + 1 + (size_t)nsm * per_sm * (size_t)n; }

int lab(int i, int N) { return i < N / 2 ? i : i - N; }

bool finite_all(const double *v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

cudaEvent_t prof_event(bym_ctx *c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch with events when tracing is on; the totals are
// gathered by prof_collect once the stream has been synchronised.
struct ProfScope {
  bym_ctx *c;
  cudaStream_t st;
  const char *name;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(bym_ctx *c_, cudaStream_t st_, const char *name_, double bytes_)
      : c(c_), st(st_), name(name_), bytes(bytes_) {
    if (c->prof) {
      a = prof_event(c);
      cudaEventRecord(a, st);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    cudaEventRecord(b, st);
    c->prof_pending.push_back({name, a, b, bytes});
  }
};

void prof_collect(bym_ctx *c) {
  for (auto &p : c->prof_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto &e = c->prof_tab[p.name];
      e.launches += 1;
      e.ms += ms;
      e.bytes += p.bytes;
    } else {
      cudaGetLastError();
    }
    c->prof_pool.push_back(p.a);
    c->prof_pool.push_back(p.b);
  }
  c->prof_pending.clear();
}

}  // namespace

// ---------------------------------------------------------------------------
// validation and sizes
// ---------------------------------------------------------------------------
int bym::validate_params(bym_ctx *c, const bym_params *p) {
  if (!p) return fail(c, BYM_E_INVAL, "params is NULL");
  if (p->ell_max < 0 || p->ell_max % 2 || p->ell_max > 8)
    return fail(c, BYM_E_UNSUPPORTED, "ell_max must be even and at most 8");
  if (p->order < 0 || p->order > 12) return fail(c, BYM_E_UNSUPPORTED, "order must be in 0..12");
  if (p->n_mesh < 8 || p->n_mesh > 1024 || p->n_mesh % 2)
    return fail(c, BYM_E_UNSUPPORTED, "n_mesh must be even and in 8..1024");
  if (p->assign != 2 && p->assign != 3) return fail(c, BYM_E_INVAL, "assign must be 2 (CIC) or 3 (TSC)");
  if (p->los < 0 || p->los > 3) return fail(c, BYM_E_INVAL, "los must be 0, 1, 2 or 3");
  if (p->los == BYM_LOS_MIDPOINT_EVEN && p->order > 4)
    return fail(c, BYM_E_UNSUPPORTED, "the parity-even midpoint form is available to order 4");
  if (p->precision != 32 && p->precision != 64) return fail(c, BYM_E_INVAL, "precision must be 32 or 64");
  if (p->norm < 0 || p->norm > 2) return fail(c, BYM_E_INVAL, "norm must be 0, 1 or 2");
  if (p->compensate != 0 && p->compensate != 1) return fail(c, BYM_E_INVAL, "compensate must be 0 or 1");
  if (p->interlace != 0 && p->interlace != 1) return fail(c, BYM_E_INVAL, "interlace must be 0 or 1");
  if (!(p->box_len > 0.0) || !std::isfinite(p->box_len) || !finite_all(p->box_lo, 3))
    return fail(c, BYM_E_INVAL, "box must be finite with box_len > 0");
  return BYM_OK;
}

int bym::validate(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                  const bym_bins *kb, const bym_bins *rb) {
  int rc = validate_params(c, p);
  if (rc) return rc;
  if (!gal || gal->n < 0 || (gal->n > 0 && !gal->xyzw)) return fail(c, BYM_E_INVAL, "bad galaxy catalog");
  if (ran && (ran->n < 0 || (ran->n > 0 && !ran->xyzw))) return fail(c, BYM_E_INVAL, "bad random catalog");
  const bool have_ran = ran && ran->n > 0;
  if (p->norm >= 1 && (!have_ran || !ran->nbar))
    return fail(c, BYM_E_INVAL, "norm = 1 or 2 needs randoms with nbar");
  for (const bym_catalog *cat : {gal, ran}) {
    if (cat && cat->n > 0 && cat->on_device && ((uintptr_t)cat->xyzw % 16))
      return fail(c, BYM_E_INVAL, "device xyzw must be 16-byte aligned");
  }
  for (const bym_bins *b : {kb, rb}) {
    if (!b) continue;
    if (!b->edges || b->nbins < 1 || b->nbins > 1024) return fail(c, BYM_E_INVAL, "bins: need 1..1024 bins");
    if (!finite_all(b->edges, b->nbins + 1) || b->edges[0] < 0.0)
      return fail(c, BYM_E_INVAL, "bins: edges must be finite and non-negative");
    for (int i = 0; i < b->nbins; ++i)
      if (!(b->edges[i + 1] > b->edges[i])) return fail(c, BYM_E_INVAL, "bins: edges must increase");
  }
  return BYM_OK;
}

static int order_key(const bym_params *p) { return p->los == BYM_LOS_YAMAMOTO ? 0 : p->order; }

static int n_fields(const bym_params *p) {
  if (p->los == BYM_LOS_YAMAMOTO) return n_even_lm(p->ell_max);
  if (p->los == BYM_LOS_BISECTOR) {
    const int J = p->ell_max + p->order / 2;
    return (J + 1) * (J + 1);
  }
  return (int)midpoint_gfields(p->ell_max, p->order, p->los == BYM_LOS_MIDPOINT_EVEN).size();
}

static bool is_midpoint(const bym_params *p) { return p->los == BYM_LOS_MIDPOINT || p->los == BYM_LOS_MIDPOINT_EVEN; }

static int n_extra_slots(const bym_params *p, bool want_pk, bool want_xi) {
  if (is_midpoint(p) && want_pk) return n_even_lm(p->ell_max);
  if (p->los == BYM_LOS_BISECTOR && want_xi) return n_even_lm(p->ell_max);
  return 0;
}

size_t bym::footprint_bytes(const bym_params *p, int64_t n_gal, int64_t n_ran, bool want_pk, bool want_xi,
                            bool cats_on_device, int chunk, bool cross) {
  const size_t N = (size_t)p->n_mesh;
  const size_t esz = p->precision == 64 ? 8 : 4;
  const size_t slot = N * N * (N + kRowPad) * esz;
  const size_t nf = (size_t)n_fields(p);
  size_t fslots = 1 + nf;                                   // delta + every field
  if (chunk > 0 && is_midpoint(p)) fslots = 2 + std::min(nf, (size_t)chunk);          // two deltas, a range
  if (chunk > 0 && p->los == BYM_LOS_BISECTOR) fslots = 1 + 2 * std::min(nf, (size_t)chunk);  // two blocks
  if (p->interlace) fslots = 2 + 2 * nf;                  // the second set on the shifted mesh
  if (cross) fslots = 2 + 2 * nf;                         // the second tracer's delta and fields
  const size_t slots = fslots + (size_t)n_extra_slots(p, want_pk, want_xi);
  size_t cats = 0;
  if (!cats_on_device) cats = (size_t)(std::max<int64_t>(n_gal, 0) + std::max<int64_t>(n_ran, 0)) * 20;
  return slots * slot + cats + (1 << 20);
}

// ---------------------------------------------------------------------------
// cuFFT plans (in place, padded real layout), shared work area
// ---------------------------------------------------------------------------
// rank 3: whole N^3 slots (batch = slots); rank 2: the (y, z) planes of slots (batch = planes)
static int get_plan(bym_ctx *c, cudaStream_t st, int N, int prec, int inverse, int batch, cufftHandle *out,
                    int rank = 3) {
  auto key = std::make_tuple(N, prec, inverse + (rank == 2 ? 2 : 0), batch);
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    *out = it->second;
    return BYM_OK;
  }
  cufftHandle h;
  if (cufftCreate(&h) != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftCreate failed");
  cufftSetAutoAllocation(h, 0);
  long long n3[3] = {N, N, N};
  long long real_emb3[3] = {N, N, N + kRowPad};          // the padded layout (kernels.cuh)
  long long cplx_emb3[3] = {N, N, (N + kRowPad) / 2};
  long long *n = rank == 2 ? n3 + 1 : n3, *real_emb = rank == 2 ? real_emb3 + 1 : real_emb3,
            *cplx_emb = rank == 2 ? cplx_emb3 + 1 : cplx_emb3;
  const long long rdist = (long long)(rank == 2 ? 1 : N) * N * (N + kRowPad);
  const long long cdist = (long long)(rank == 2 ? 1 : N) * N * ((N + kRowPad) / 2);
  cufftType type = prec == 64 ? (inverse ? CUFFT_Z2D : CUFFT_D2Z) : (inverse ? CUFFT_C2R : CUFFT_R2C);
  size_t work = 0;
  cufftResult r;
  if (!inverse)
    r = cufftMakePlanMany64(h, rank, n, real_emb, 1, rdist, cplx_emb, 1, cdist, type, batch, &work);
  else
    r = cufftMakePlanMany64(h, rank, n, cplx_emb, 1, cdist, real_emb, 1, rdist, type, batch, &work);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return fail(c, BYM_E_CUDA, "cufftMakePlanMany failed (" + std::to_string((int)r) + ")");
  }
  if (work > c->fft_work_size) {
    // grow the work area in the order of the request's stream (every use of it is on
    // that stream, and the previous request finished before this one started): no
    // device-wide synchronisation, so other contexts (serving slots) keep running
    if (c->fft_work) cudaFreeAsync(c->fft_work, st);
    c->fft_work = nullptr;
    c->fft_work_size = 0;
    if (cudaMallocAsync(&c->fft_work, work, st) != cudaSuccess) {
      cudaGetLastError();
      cufftDestroy(h);
      return fail(c, BYM_E_NOMEM, "cuFFT work area allocation failed");
    }
    c->fft_work_size = work;
  }
  c->plans[key] = h;
  *out = h;
  return BYM_OK;
}

static const Tune &tune_for(bym_ctx *c, int N, int prec, int los) {
  static const Tune kDefault;
  auto it = c->tune.find(std::make_tuple(N, prec, los));
  return it == c->tune.end() ? kDefault : it->second;
}

// Which FFT path a request takes: 0 cuFFT 3D transforms; 1 cuFFT 2D transforms of the
// (y, z) planes with the library's x pass (and the convolution product fused into
// it); 2 cuFFT 2D plane transforms and cuFFT 1D transforms along x (any mesh and
// precision); 8 / 16 the library's two-pass transforms with 8- / 16-CTA plane clusters.
// FFT path of a request: 0 cuFFT 3D, 1 cuFFT planes + library x pass, 2 cuFFT planes + cuFFT x,
// 3 library z, y and x passes, 8 / 16 library two-pass (cluster plane pass + x pass)
static int fft_kind(const bym_ctx *c, int N, int prec, const Tune &tn) {
  if (c->fft_mode == 5) return 2;
  if (!native_fft_supported(N, prec)) return (c->fft_mode == 2 && tn.native == 2) ? 2 : 0;
  switch (c->fft_mode) {
    case 0: return 0;
    case 1: return 8;
    case 3: return 16;
    case 4: return 1;
    case 6: return 3;
    default:
      if (tn.native < 0) return 3;   // untuned: the library's z, y and x passes
      return (tn.native == 1 || tn.native == 2 || tn.native == 3 || tn.native == 8 || tn.native == 16) ? tn.native
                                                                                                       : 0;
  }
}

// cuFFT 1D C2C transforms along x of every (ky, kz) column of one slot's half spectrum, the
// padding column included (stride N (N + kRowPad) / 2 complex, in place); the sign is chosen at
// execution
static int get_xplan(bym_ctx *c, cudaStream_t st, int N, int prec, cufftHandle *out) {
  auto key = std::make_tuple(N, prec, 6, 1);
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    *out = it->second;
    return BYM_OK;
  }
  cufftHandle h;
  if (cufftCreate(&h) != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftCreate failed");
  cufftSetAutoAllocation(h, 0);
  long long n[1] = {N}, emb[1] = {N};
  const long long H2 = (long long)N * ((N + kRowPad) / 2);
  size_t work = 0;
  const cufftResult r = cufftMakePlanMany64(h, 1, n, emb, H2, 1, emb, H2, 1, prec == 64 ? CUFFT_Z2Z : CUFFT_C2C, H2,
                                            &work);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return fail(c, BYM_E_CUDA, "cufftMakePlanMany (x) failed (" + std::to_string((int)r) + ")");
  }
  if (work > c->fft_work_size) {   // as in get_plan: grown in the order of the request's stream
    if (c->fft_work) cudaFreeAsync(c->fft_work, st);
    c->fft_work = nullptr;
    c->fft_work_size = 0;
    if (cudaMallocAsync(&c->fft_work, work, st) != cudaSuccess) {
      cudaGetLastError();
      cufftDestroy(h);
      return fail(c, BYM_E_NOMEM, "cuFFT work area allocation failed");
    }
    c->fft_work_size = work;
  }
  c->plans[key] = h;
  *out = h;
  return BYM_OK;
}

// Forward plane transforms of painted or generated fields over the x planes [x0, x0 + np) only
// (np = 0: all): the other planes of such a field are zero, and so are their transforms.
struct XRange {
  int x0 = 0, np = 0;
  int y0 = 0, ny = 0;  // the rows y in [y0, y0 + ny) of every plane (ny = 0: all) hold the painted values
  bool rows = false;   // the x pass reads only the range's rows too (library x pass), so the other
                       // planes of a field slot need no zero-fill
};

// cuFFT 2D transforms of the planes of slots [first, first + count), tn.fft_batch slots per call;
// forward with a plane range: one call per slot over the range's planes
static cufftResult plane_exec(cufftHandle h, int prec, int inverse, char *ptr) {
  if (prec == 64)
    return inverse ? cufftExecZ2D(h, (cufftDoubleComplex *)ptr, (cufftDoubleReal *)ptr)
                   : cufftExecD2Z(h, (cufftDoubleReal *)ptr, (cufftDoubleComplex *)ptr);
  return inverse ? cufftExecC2R(h, (cufftComplex *)ptr, (cufftReal *)ptr)
                 : cufftExecR2C(h, (cufftReal *)ptr, (cufftComplex *)ptr);
}

static int fft_planes(bym_ctx *c, cudaStream_t st, int inverse, int N, void *base, size_t slot_bytes, int first,
                      int count, const Tune &tn, const XRange *xr = nullptr, int prec = 32) {
  if (xr && xr->np > 0 && !inverse) {
    const size_t plane_bytes = slot_bytes / N;
    for (int i = 0; i < count; ++i) {
      cufftHandle h;
      int rc = get_plan(c, st, N, prec, 0, xr->np, &h, 2);
      if (rc) return rc;
      cufftSetStream(h, st);
      cufftSetWorkArea(h, c->fft_work);
      char *ptr = (char *)base + (size_t)(first + i) * slot_bytes + (size_t)xr->x0 * plane_bytes;
      if (plane_exec(h, prec, 0, ptr) != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftExec (plane range) failed");
    }
    return BYM_OK;
  }
  for (int done = 0; done < count;) {
    const int b = std::min(std::max(tn.fft_batch, 1), count - done);
    cufftHandle h;
    int rc = get_plan(c, st, N, prec, inverse, b * N, &h, 2);
    if (rc) return rc;
    cufftSetStream(h, st);
    cufftSetWorkArea(h, c->fft_work);
    char *ptr = (char *)base + (size_t)(first + done) * slot_bytes;
    const cufftResult r = plane_exec(h, prec, inverse, ptr);
    if (r != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftExec (planes) failed (" + std::to_string((int)r) + ")");
    done += b;
  }
  return BYM_OK;
}

// The (y, z) plane transforms of FP32 512^3 slots for the library's x pass: cuFFT 2D transforms
// (kind 1) or the library's z and y passes (kind 3); forward over the plane range (and, kind 3,
// the row range) of xr when given
static int plane_transforms(bym_ctx *c, cudaStream_t st, int kind, int inverse, int N, void *base, size_t slot_bytes,
                            int first, int count, const Tune &tn, const XRange *xr) {
  const bool rng = !inverse && xr && xr->np > 0, yr = !inverse && xr && xr->ny > 0;
  const int x0 = rng ? xr->x0 : 0, x1 = rng ? xr->x0 + xr->np : N;
  const int y0 = yr ? xr->y0 : 0, y1 = yr ? xr->y0 + xr->ny : N;
  if (kind == 1) {
    ProfScope ps(c, st, inverse ? "cufft_planes_c2r" : "cufft_planes_r2c", count * 2.0 * 4.0 * (double)(x1 - x0) * N * N);
    return fft_planes(c, st, inverse, N, base, slot_bytes, first, count, tn, inverse ? nullptr : xr);
  }
  // z pass: the rows it transforms, read and written; y pass: the rows it reads, every row written
  const double ny = y1 - y0, np = x1 - x0, row = 2.0 * 4.0 * (N / 2 + 1);
  const long long sr = (long long)(slot_bytes / 4);
  cudaError_t e = cudaSuccess;
  auto zp = [&]() {
    ProfScope ps(c, st, inverse ? "fft_native_z_inv" : "fft_native_z_fwd", count * 2.0 * np * ny * row);
    e = native_fft_zpass(inverse, (float *)base, sr, first, count, st, x0, x1, y0, y1);
  };
  auto yp = [&]() {
    ProfScope ps(c, st, inverse ? "fft_native_y_inv" : "fft_native_y_fwd", count * np * (ny + N) * row);
    e = native_fft_ypass(inverse, (float *)base, sr, first, count, st, x0, x1, y0, y1);
  };
  if (!inverse) {
    zp();
    if (e == cudaSuccess) yp();
  } else {
    yp();
    if (e == cudaSuccess) zp();
  }
  return e == cudaSuccess ? BYM_OK : fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
}

static int fft_slots(bym_ctx *c, cudaStream_t st, int prec, int inverse, int N, void *base, size_t slot_bytes,
                     int first, int count, const Tune &tn, const XRange *xr = nullptr) {
  const double esz = prec == 64 ? 8.0 : 4.0;
  const int kind = fft_kind(c, N, prec, tn);
  if (kind == 2) {   // cuFFT plane transforms (forward over the occupied planes), cuFFT along x
    const double np = !inverse && xr && xr->np > 0 ? xr->np : N;
    if (!inverse) {
      ProfScope ps(c, st, "cufft_planes_r2c", count * 2.0 * esz * np * N * N);
      TRY_RC(fft_planes(c, st, 0, N, base, slot_bytes, first, count, tn, xr, prec));
    }
    {
      ProfScope ps(c, st, inverse ? "cufft_x_inv" : "cufft_x_fwd", count * 4.0 * esz * N * N * (N / 2 + 1));
      cufftHandle h;
      TRY_RC(get_xplan(c, st, N, prec, &h));
      cufftSetStream(h, st);
      cufftSetWorkArea(h, c->fft_work);
      for (int i = 0; i < count; ++i) {
        char *ptr = (char *)base + (size_t)(first + i) * slot_bytes;
        const int dir = inverse ? CUFFT_INVERSE : CUFFT_FORWARD;
        const cufftResult r = prec == 64 ? cufftExecZ2Z(h, (cufftDoubleComplex *)ptr, (cufftDoubleComplex *)ptr, dir)
                                         : cufftExecC2C(h, (cufftComplex *)ptr, (cufftComplex *)ptr, dir);
        if (r != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftExec (x) failed (" + std::to_string((int)r) + ")");
      }
    }
    if (inverse) {
      ProfScope ps(c, st, "cufft_planes_c2r", count * 2.0 * esz * (double)N * N * N);
      TRY_RC(fft_planes(c, st, 1, N, base, slot_bytes, first, count, tn, nullptr, prec));
    }
    return BYM_OK;
  }
  if (kind) {
    cudaError_t e = native_fft_prepare();
    if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
    const long long sr = (long long)(slot_bytes / 4);
    const double cplx = 2.0 * esz * (double)N * N * (N / 2 + 1);
    if (kind == 1 || kind == 3) {   // cuFFT or the library's passes over the (y, z) planes, the library's x pass
      if (!inverse) TRY_RC(plane_transforms(c, st, kind, 0, N, base, slot_bytes, first, count, tn, xr));
      {
        // forward with a plane range: the rows outside it are zero and are not read
        const bool rng = !inverse && xr && xr->np > 0;
        const double rd = rng ? (double)xr->np / N : 1.0;
        ProfScope ps(c, st, inverse ? "fft_native_x_inv" : "fft_native_x_fwd", count * (1.0 + rd) * cplx);
        e = native_fft_xpass(inverse ? 1 : 0, (float *)base, sr, first, count, nullptr, nullptr, nullptr, st,
                             rng ? xr->x0 : 0, rng ? xr->x0 + xr->np : N);
      }
      if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
      if (inverse) TRY_RC(plane_transforms(c, st, kind, 1, N, base, slot_bytes, first, count, tn, nullptr));
      return BYM_OK;
    }
    {
      ProfScope ps(c, st, inverse ? "fft_native_c2r" : "fft_native_r2c", count * 2.0 * esz * (double)N * N * N);
      e = inverse ? native_fft_inverse((float *)base, sr, first, count, kind, st)
                  : native_fft_forward((float *)base, sr, first, count, kind, st);
    }
    if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
    return BYM_OK;
  }
  ProfScope ps(c, st, inverse ? "cufft_c2r" : "cufft_r2c", count * 2.0 * esz * (double)N * N * N);
  for (int done = 0; done < count;) {
    const int b = std::min(std::max(tn.fft_batch, 1), count - done);
    cufftHandle h;
    int rc = get_plan(c, st, N, prec, inverse, b, &h);
    if (rc) return rc;
    cufftSetStream(h, st);
    cufftSetWorkArea(h, c->fft_work);
    char *ptr = (char *)base + (size_t)(first + done) * slot_bytes;
    cufftResult r;
    if (prec == 64)
      r = inverse ? cufftExecZ2D(h, (cufftDoubleComplex *)ptr, (cufftDoubleReal *)ptr)
                  : cufftExecD2Z(h, (cufftDoubleReal *)ptr, (cufftDoubleComplex *)ptr);
    else
      r = inverse ? cufftExecC2R(h, (cufftComplex *)ptr, (cufftReal *)ptr)
                  : cufftExecR2C(h, (cufftReal *)ptr, (cufftComplex *)ptr);
    if (r != CUFFT_SUCCESS) return fail(c, BYM_E_CUDA, "cufftExec failed (" + std::to_string((int)r) + ")");
    done += b;
  }
  return BYM_OK;
}

// The convolution steps of the midpoint series for fields [first, first + count)
// (slots hold real fields; D = slot 0 holds delta's half spectrum): forward,
// times conj(D) scale W^-2, inverse.  With the library's kernels the product
// sits between the forward and inverse x passes.
template <typename T, typename T2>
static int convolve_fields(bym_ctx *c, cudaStream_t st, int prec, int N, void *slots, size_t slot_bytes, int first,
                           int count, const double *scale, const T *invw, const Tune &tn,
                           const XRange *xr = nullptr) {
  const int kind = fft_kind(c, N, prec, tn);
  const double esz = sizeof(T), n3 = (double)N * N * N, cplx = 2.0 * esz * N * N * (N / 2 + 1);
  const long long slot_reals = (long long)(slot_bytes / sizeof(T));
  if (kind && kind != 2) {
    cudaError_t e = native_fft_prepare();
    if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
    if (kind == 1 || kind == 3) {
      TRY_RC(plane_transforms(c, st, kind, 0, N, slots, slot_bytes, first, count, tn, xr));
      {
        // read every F once over its occupied rows and D once (each D tile serves all fields of the
        // launch), write F
        const bool rng = xr && xr->np > 0;
        const double rd = rng ? (double)xr->np / N : 1.0;
        ProfScope ps(c, st, "fft_native_x_convolve", (count * (1.0 + rd) + 1.0) * cplx);
        e = native_fft_xpass(2, (float *)slots, slot_reals, first, count, (const float *)slots, scale,
                             (const float *)invw, st, rng ? xr->x0 : 0, rng ? xr->x0 + xr->np : N);
      }
      if (e == cudaSuccess) TRY_RC(plane_transforms(c, st, kind, 1, N, slots, slot_bytes, first, count, tn, nullptr));
    } else {
      ProfScope ps(c, st, "fft_native_convolve", count * (2.0 * n3 * esz + cplx));
      e = native_fft_convolve((float *)slots, slot_reals, first, count, (const float *)slots, scale,
                              (const float *)invw, kind, st);
    }
    if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("native FFT: ") + cudaGetErrorString(e));
    return BYM_OK;
  }
  TRY_RC(fft_slots(c, st, prec, 0, N, slots, slot_bytes, first, count, tn, xr));
  {
    ProfScope ps(c, st, "spec_mul", (2.0 * count + 1.0) * cplx);
    launch_spec_mul<T, T2>((T2 *)((char *)slots + (size_t)first * slot_bytes), slot_reals / 2, count,
                           (const T2 *)slots, N, scale, invw, c->nsm * tn.per_sm_spec / 8, st);
  }
  return fft_slots(c, st, prec, 1, N, slots, slot_bytes, first, count, tn);
}

// ---------------------------------------------------------------------------
// shell geometry: bin look-up tables over |n|^2 and per-bin counts / means
// ---------------------------------------------------------------------------
static std::string geom_key(int N, double L, const bym_bins *b, char kind) {
  std::ostringstream o;
  o << kind << N << ':';
  o.write((const char *)&L, sizeof L);
  o.write((const char *)b->edges, sizeof(double) * (b->nbins + 1));
  return o.str();
}

static std::vector<int> bin_lut(int N, double unit, const bym_bins *b) {
  const int h = N / 2;
  const long long n2max = 3LL * h * h;
  std::vector<int> lut((size_t)n2max + 1, -1);
  const double *e = b->edges;
  for (long long n2 = 1; n2 <= n2max; ++n2) {
    const double mag = unit * std::sqrt((double)n2);
    const double *u = std::upper_bound(e, e + b->nbins + 1, mag);
    const long long bin = (long long)(u - e) - 1;
    if (bin >= 0 && bin < b->nbins) lut[(size_t)n2] = (int)bin;
  }
  return lut;
}

static int get_geom(bym_ctx *c, const KernelSet &ks, int N, double L, const bym_bins *b, char kind,
                    cudaStream_t st, Geom **out) {
  auto &cache = kind == 'k' ? c->kgeo : c->rgeo;
  const std::string key = geom_key(N, L, b, kind);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = &it->second;
    return BYM_OK;
  }
  Geom g;
  g.nbins = b->nbins;
  const double h = L / N;
  const double unit = kind == 'k' ? 2.0 * M_PI / L : h;
  std::vector<int> lut = bin_lut(N, unit, b);
  if (cudaMalloc(&g.lut, lut.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "bin table allocation failed");
  }
  cudaMemcpy(g.lut, lut.data(), lut.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (kind == 'r') {
    int jm = (int)std::floor(b->edges[b->nbins] / h) + 1;
    g.full = (2 * jm + 1 > N) ? 1 : 0;
    g.jm = g.full ? N / 2 : jm;
  }
  double *sums = nullptr;
  if (cudaMalloc(&sums, sizeof(double) * sums_doubles(2 * b->nbins, c->nsm, 4)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "geometry allocation failed");
  }
  cudaMemsetAsync(sums, 0, sizeof(double) * (2 * b->nbins + 1), st);
  cudaError_t e;
  const size_t smem = sums_smem(2 * b->nbins);
  if (kind == 'k') {
    const long long work = (long long)N * N * (N / 2 + 1);
    e = launch(ks.kgeom, grid_of(work, c->nsm, 4), 256, smem, st, N, (const int *)g.lut, b->nbins, unit, sums);
  } else {
    const int Lc = g.full ? N : 2 * g.jm + 1;
    const long long work = (long long)Lc * Lc * Lc;
    e = launch(ks.rgeom, grid_of(work, c->nsm, 4), 256, smem, st, N, g.jm, g.full, (const int *)g.lut, b->nbins, h,
               sums);
  }
  std::vector<double> hs(2 * b->nbins);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), sums, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sums);
  if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("geometry kernel: ") + cudaGetErrorString(e));
  g.count.resize(b->nbins);
  g.mean.resize(b->nbins);
  for (int i = 0; i < b->nbins; ++i) {
    g.count[i] = (int64_t)std::llround(hs[2 * i]);
    g.mean[i] = g.count[i] > 0 ? hs[2 * i + 1] / hs[2 * i] : 0.0;
  }
  if (kind == 'k') {
    // count = sum over the binned half-spectrum modes of their weight (1 on the kz = 0 and
    // kz = N/2 planes, 2 elsewhere): half modes = (count + weight-1 modes) / 2
    long long total = 0, w1 = 0;
    for (int i = 0; i < b->nbins; ++i) total += g.count[i];
    for (int iz : {0, N / 2})
      for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy) {
          const long long nx = ix < N / 2 ? ix : ix - N, ny = iy < N / 2 ? iy : iy - N, nz = iz;
          if (lut[(size_t)(nx * nx + ny * ny + nz * nz)] >= 0) ++w1;
        }
    g.half_binned = (total + w1) / 2;
  }
  auto res = cache.emplace(key, std::move(g));
  *out = &res.first->second;
  return BYM_OK;
}

// A table of -1 (no k bin) for requests that need X(k) but no P.
static int get_null_kgeom(bym_ctx *c, int N, Geom **out) {
  const std::string key = "null" + std::to_string(N);
  auto it = c->kgeo.find(key);
  if (it != c->kgeo.end()) {
    *out = &it->second;
    return BYM_OK;
  }
  Geom g;
  g.nbins = 1;
  const size_t n = 3 * (size_t)(N / 2) * (N / 2) + 1;
  std::vector<int> lut(n, -1);
  if (cudaMalloc(&g.lut, n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "bin table allocation failed");
  }
  cudaMemcpy(g.lut, lut.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  auto res = c->kgeo.emplace(key, std::move(g));
  *out = &res.first->second;
  return BYM_OK;
}

// Device bytes a request may still take: free memory plus what the stream-ordered
// pool holds unused, less the given headroom (FFT work areas and small buffers).
size_t bym::device_available(bym_ctx *c, size_t headroom) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
      free_b += (size_t)(reserved - used);
  }
  return free_b > headroom ? free_b - headroom : 0;
}

// ---------------------------------------------------------------------------
// one request
// ---------------------------------------------------------------------------
// A request enqueued without waiting (CUDA-graph batches): pinned host areas for the
// small uploads and for the results, and what the host step after the launch needs.
struct Pending {
  double *host = nullptr;       // pinned: [8 stats][NL * nbk P sums][NL * nbr xi sums]
  char *stage = nullptr;        // pinned: [nf scale factors (double)][n_mesh 1/W (T)][n_mesh phases (T2)]
  size_t host_len = 0, stage_len = 0;
  Geom *kg = nullptr, *rg = nullptr;
  int NL = 0, nbk = 0, nbr = 0;
  double h = 0.0;
};

// Host normalisation of the FP64 sums (Sec. 2 with the readings of the library's
// normalisation: P = 4 pi / A * bin mean, xi = 4 pi / (A V_cell) * bin mean).
// cross: hstats holds 16 sums, tracer B's at [8, 16); A = sqrt(A_A A_B).  pk_scale multiplies
// the P sums (the Yamamoto cross spectrum adds its two endpoint terms without the 1/2).
static int finish_results(bym_ctx *c, const Request &rq, const double *hstats, const double *hk, const double *hr,
                          const Geom *kg, const Geom *rg, int NL, int nbk, int nbr, double h, bool cross = false,
                          double pk_scale = 1.0) {
  const bym_params *p = rq.p;
  if (native_fft_fault(c->device))
    return fail(c, BYM_E_CUDA, "a 512^3 x pass gave up waiting for a tile copy on this device; results are invalid");
  const double bad = hstats[3] + (cross ? hstats[11] : 0.0);
  if (bad > 0.0)
    return fail(c, BYM_E_OUT_OF_BOX, std::to_string((long long)bad) + " objects lie outside the box or are not finite");
  if (rq.alpha) *rq.alpha = hstats[1] != 0.0 ? hstats[0] / hstats[1] : 0.0;
  double A = 1.0, vcell = 1.0;
  if (p->norm >= 1) {
    const double alpha = hstats[0] / hstats[1];
    A = alpha * hstats[2];
    if (cross) A = std::sqrt(A * (hstats[8] / hstats[9]) * hstats[10]);
    vcell = h * h * h;
    if (!(A > 0.0) || !std::isfinite(A)) return fail(c, BYM_E_INVAL, "FKP normalisation A is not positive");
  }
  // norm 2: xi as raw sums here, divided by the random-random count afterwards
  const double xden = p->norm == 2 ? 1.0 : A * vcell;
  const double four_pi = 4.0 * M_PI;
  if (rq.kb) {
    for (int l = 0; l < NL; ++l)
      for (int b = 0; b < nbk; ++b)
        rq.pk[l * nbk + b] =
            kg->count[b] > 0 ? pk_scale * four_pi / A * hk[(size_t)b * NL + l] / (double)kg->count[b] : 0.0;
    if (rq.kmean) std::copy(kg->mean.begin(), kg->mean.end(), rq.kmean);
    if (rq.nmodes) std::copy(kg->count.begin(), kg->count.end(), rq.nmodes);
  }
  if (rq.rb) {
    for (int l = 0; l < NL; ++l)
      for (int b = 0; b < nbr; ++b)
        rq.xi[l * nbr + b] =
            rg->count[b] > 0 ? four_pi / xden * hr[(size_t)b * NL + l] / (double)rg->count[b] : 0.0;
    if (rq.rmean) std::copy(rg->mean.begin(), rg->mean.end(), rq.rmean);
    if (rq.ncells) std::copy(rg->count.begin(), rg->count.end(), rq.ncells);
  }
  return BYM_OK;
}

// The x planes that hold painted values in the delta slots given (their union), and the rows y
// that do, each rounded out to a multiple of 32 (so that few plan sizes arise, and the tiles of
// the library's passes line up); waits for the stream.  Leaves *out at "every plane" / "every
// row" when nothing was painted or a range spans the mesh.
template <typename T>
static int plane_range(bym_ctx *c, cudaStream_t st, DevBufs &buf, const std::vector<const T *> &deltas, int N,
                       XRange *out) {
  int *d = nullptr;
  if (buf.alloc((void **)&d, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "plane range allocation failed");
  }
  const int init[4] = {N, -1, N, -1};
  int h[4] = {N, -1, N, -1};
  cudaError_t e = cudaMemcpyAsync(d, init, sizeof init, cudaMemcpyHostToDevice, st);
  {
    ProfScope ps(c, st, "plane_range", (double)deltas.size() * N * N * (N + kRowPad) * sizeof(T));
    for (const T *p : deltas)
      if (e == cudaSuccess) {
        launch_plane_range<T>(p, N, d, st);
        e = cudaGetLastError();
      }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("plane range: ") + cudaGetErrorString(e));
  if (h[1] < h[0] || h[0] < 0 || h[1] >= N || h[3] < h[2] || h[2] < 0 || h[3] >= N) return BYM_OK;
  // whole blocks of 32 planes and rows (the passes move tiles in boxes of 32 rows)
  const int x0 = h[0] / 32 * 32, x1 = std::min(N, (h[1] + 32) / 32 * 32), np = x1 - x0;
  const int y0 = h[2] / 32 * 32, y1 = std::min(N, (h[3] + 32) / 32 * 32), ny = y1 - y0;
  if (ny < N) {
    out->y0 = y0;
    out->ny = ny;
  }
  if (np >= N) return BYM_OK;
  out->x0 = x0;
  out->np = np;
  return BYM_OK;
}

// pd == nullptr: run the request and wait.  pd != nullptr: enqueue it on st (nothing
// waits; uploads come from pd->stage, results land in pd->host) for finish_results
// after the stream (or the graph it was captured into) has run; catalogs must then be
// device catalogs, and every cache the request uses (kernels, geometry, FFT plans and
// work area) must exist already, as they do after one run of a request of that shape.
template <typename T, typename T2>
static int run_typed(bym_ctx *c, const Request &rq, cudaStream_t st, Pending *pd = nullptr) {
  const bym_params *p = rq.p;
  const int N = p->n_mesh;
  const bool want_pk = rq.kb != nullptr, want_xi = rq.rb != nullptr;
  std::string jerr;
  auto ks = get_kernels(JitKey{p->los, p->ell_max, order_key(p), p->precision}, jerr);
  if (!ks) return fail(c, BYM_E_CUDA, jerr);
  const KernelSet &K = *ks;
  const Tune &tn = tune_for(c, N, p->precision, p->los);
  const int nf = (int)K.fields.size();
  const int nlm = K.n_lm, NL = K.n_ell;
  const int nextra = n_extra_slots(p, want_pk, want_xi);
  const long long slot_reals = (long long)N * N * (N + kRowPad);
  const long long cslot = slot_reals / 2;
  const size_t slot_bytes = (size_t)slot_reals * sizeof(T);
  const double h = p->box_len / N, inv_h = N / p->box_len, inv_r0 = 1.0 / p->box_len;

  // midpoint g fields streamed in ranges when forced, or when the whole set does not fit
  const bool cross = rq.gal_b != nullptr;
  const bool cats_dev = rq.gal->on_device && (!rq.ran || rq.ran->on_device) &&
                        (!cross || (rq.gal_b->on_device && (!rq.ran_b || rq.ran_b->on_device)));
  const int64_t ngal = rq.gal->n + (cross ? rq.gal_b->n : 0);
  const int64_t nran = (rq.ran ? rq.ran->n : 0) + (cross && rq.ran_b ? rq.ran_b->n : 0);
  int chunk = 0;
  if (p->interlace && c->field_chunk > 0 && p->los != BYM_LOS_YAMAMOTO)
    return fail(c, BYM_E_UNSUPPORTED, "interlacing keeps every field resident: no field ranges");
  if (cross && (p->interlace || p->norm == 2 || (c->field_chunk > 0 && p->los != BYM_LOS_YAMAMOTO)))
    return fail(c, BYM_E_UNSUPPORTED, "cross spectra: no interlacing, no norm 2, both field sets resident");
  if (cross && pd) return fail(c, BYM_E_INVAL, "cross spectra are not enqueued");
  if (!p->interlace && !cross && (is_midpoint(p) || p->los == BYM_LOS_BISECTOR)) {
    if (c->field_chunk > 0) {
      chunk = std::min(c->field_chunk, nf);
    } else {
      // without a budget: free memory less room for the FFT work area (up to a batch of transforms)
      const size_t head = (size_t)(std::max(tn.fft_batch, 1) + 1) * slot_bytes;
      const size_t avail = c->budget ? c->budget : device_available(c, head);
      if (footprint_bytes(p, ngal, nran, want_pk, want_xi, cats_dev) > avail)
        for (int m = nf - 1; m >= 1 && !chunk; --m)
          if (footprint_bytes(p, ngal, nran, want_pk, want_xi, cats_dev, m) <= avail) chunk = m;
    }
  }
  if (c->budget && footprint_bytes(p, ngal, nran, want_pk, want_xi, cats_dev, chunk, cross) > c->budget)
    return fail(c, BYM_E_NOMEM, "request exceeds the context's HBM budget");
  cudaKernel_t kx = nullptr;   // bisector cross contraction
  if (cross && p->los == BYM_LOS_BISECTOR) {
    kx = get_cross_kernel(JitKey{p->los, p->ell_max, order_key(p), p->precision}, jerr);
    if (!kx) return fail(c, BYM_E_CUDA, jerr);
  }
  std::shared_ptr<ChunkSet> CK;
  if (chunk) {
    CK = get_chunk_kernels(JitKey{p->los, p->ell_max, order_key(p), p->precision}, chunk, jerr);
    if (!CK) return fail(c, BYM_E_CUDA, jerr);
  }

  Geom *kg = nullptr, *rg = nullptr;
  int rc;
  if (want_pk && (rc = get_geom(c, K, N, p->box_len, rq.kb, 'k', st, &kg))) return rc;
  if (want_xi && (rc = get_geom(c, K, N, p->box_len, rq.rb, 'r', st, &rg))) return rc;
  if (!kg && p->los == BYM_LOS_BISECTOR && (rc = get_null_kgeom(c, N, &kg))) return rc;

  DevBufs buf(st);
  auto alloc = [&](void **ptr, size_t bytes) -> int {
    if (buf.alloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, BYM_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return BYM_OK;
  };
#define TRY(x)                  \
  do {                          \
    int rc_ = (x);              \
    if (rc_) return rc_;        \
  } while (0)
#define CUDA_TRY(x)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return fail(c, BYM_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

  // catalogs: galaxies and randoms of tracer A, then of tracer B (cross spectra)
  const float4 *cat4[4] = {nullptr, nullptr, nullptr, nullptr};
  const float *catnb[4] = {nullptr, nullptr, nullptr, nullptr};
  const bym_catalog *cats[4] = {rq.gal, rq.ran, cross ? rq.gal_b : nullptr, cross ? rq.ran_b : nullptr};
  long long catn[4];
  for (int w = 0; w < 4; ++w) catn[w] = cats[w] ? cats[w]->n : 0;
  for (int w = 0; w < 4; ++w) {
    const bym_catalog *cat = cats[w];
    if (!cat || cat->n <= 0) continue;
    if (cat->on_device) {
      cat4[w] = (const float4 *)cat->xyzw;
      catnb[w] = cat->nbar;
    } else if (pd) {
      return fail(c, BYM_E_INVAL, "an enqueued request needs device catalogs");
    } else {
      void *d4 = nullptr;
      TRY(alloc(&d4, (size_t)cat->n * 16));
      CUDA_TRY(cudaMemcpyAsync(d4, cat->xyzw, (size_t)cat->n * 16, cudaMemcpyHostToDevice, st));
      cat4[w] = (const float4 *)d4;
      if (cat->nbar) {
        void *dn = nullptr;
        TRY(alloc(&dn, (size_t)cat->n * 4));
        CUDA_TRY(cudaMemcpyAsync(dn, cat->nbar, (size_t)cat->n * 4, cudaMemcpyHostToDevice, st));
        catnb[w] = (const float *)dn;
      }
    }
  }

  double *stats = nullptr, *ksum = nullptr, *rsum = nullptr, *scale = nullptr;
  T *invw = nullptr;
  TRY(alloc((void **)&stats, 16 * sizeof(double)));    // [0, 8) tracer A, [8, 16) tracer B
  CUDA_TRY(cudaMemsetAsync(stats, 0, 16 * sizeof(double), st));
  const int nbk = want_pk ? rq.kb->nbins : 1, nbr = want_xi ? rq.rb->nbins : 1;
  // shell sums, their ticket counter (zeroed) and room for one total per block
  TRY(alloc((void **)&ksum, sizeof(double) * sums_doubles(NL * nbk, c->nsm, std::max(tn.per_sm_k, 1))));
  TRY(alloc((void **)&rsum, sizeof(double) * sums_doubles(NL * nbr, c->nsm, 4)));
  CUDA_TRY(cudaMemsetAsync(ksum, 0, sizeof(double) * (NL * nbk + 1), st));
  CUDA_TRY(cudaMemsetAsync(rsum, 0, sizeof(double) * (NL * nbr + 1), st));
  if (p->compensate) {
    std::vector<T> w(N);
    for (int i = 0; i < N; ++i) {
      const double x = M_PI * lab(i, N) / N;
      const double s = x == 0.0 ? 1.0 : std::sin(x) / x;
      w[i] = (T)(1.0 / std::pow(s, p->assign));
    }
    TRY(alloc((void **)&invw, sizeof(T) * N));
    const void *src = w.data();
    if (pd) {
      T *dst = (T *)(pd->stage + sizeof(double) * (size_t)nf);
      std::copy(w.begin(), w.end(), dst);
      src = dst;
    }
    CUDA_TRY(cudaMemcpyAsync(invw, src, sizeof(T) * N, cudaMemcpyHostToDevice, st));
  }
  {
    std::vector<double> sc(nf);
    const double inv_n3 = 1.0 / ((double)N * N * N);
    for (int i = 0; i < nf; ++i) {
      const double sign = (is_midpoint(p) && (K.fields[i].J % 2)) ? -1.0 : 1.0;
      sc[i] = sign * inv_n3;
    }
    TRY(alloc((void **)&scale, sizeof(double) * std::max(nf, 1)));
    const void *src = sc.data();
    if (pd) {
      std::copy(sc.begin(), sc.end(), (double *)pd->stage);
      src = pd->stage;
    }
    CUDA_TRY(cudaMemcpyAsync(scale, src, sizeof(double) * nf, cudaMemcpyHostToDevice, st));
  }

  // mesh slots: [0] delta, [1, 1+nf) fields, [1+nf, 1+nf+nextra) H or X;
  // streamed: [0] delta, [1] a real copy of delta, [2, 2+chunk) one field range, then H
  const bool bis_blocks = chunk && p->los == BYM_LOS_BISECTOR;
  const int fbase = (chunk && !bis_blocks) ? 2 : 1;
  const int nfs = !chunk ? nf : (bis_blocks ? 2 * chunk : chunk), xbase = fbase + nfs;
  // interlacing: [ibase] delta on the shifted mesh, then its field set
  const bool il = p->interlace != 0;
  const int ibase = xbase + nextra;
  // cross spectra: [cbase] tracer B's delta, then its field set
  const int cbase = ibase + (il ? 1 + nf : 0);
  const int nslots = cbase + (cross ? 1 + nf : 0);
  T *slots = nullptr;
  TRY(alloc((void **)&slots, (size_t)nslots * slot_bytes));
  auto slot_r = [&](int i) { return slots + (long long)i * slot_reals; };
  auto slot_c = [&](int i) { return (T2 *)(slots + (long long)i * slot_reals); };
  // painted slots (delta, the interlaced and the second tracer's delta) need no zero-fill: the
  // painter writes every cell

  // norms and painting
  const double esz = (double)sizeof(T), n3 = (double)N * N * N, nhalf = (double)N * N * (N / 2 + 1);
  double *npart = nullptr;
  TRY(alloc((void **)&npart, norm_scratch_bytes(c->nsm)));
  for (int w = 0; w < 4; ++w)
    if (cat4[w]) {
      ProfScope ps(c, st, "norm_reduce", catn[w] * ((w & 1) ? 20.0 : 16.0));
      launch_norm_reduce(cat4[w], catnb[w], catn[w], w & 1, p->box_lo, inv_h, N, stats + 8 * (w >> 1), npart, c->nsm,
                         st, p->precision);
    }
  {
    void *pscr = nullptr;
    TRY(alloc(&pscr, paint_scratch_bytes(N, std::max(catn[0] + catn[1], catn[2] + catn[3]))));
    for (int t = 0; t < (cross ? 2 : 1); ++t) {
      const int w = 2 * t;
      ProfScope ps(c, st, "paint", (catn[w] + catn[w + 1]) * 16.0 + n3 * esz);
      CUDA_TRY(launch_paint<T>(cat4[w], catn[w], cat4[w + 1], catn[w + 1], stats + 8 * t, slot_r(t ? cbase : 0), N,
                               p->box_lo, inv_h, p->assign, pscr, c->nsm, st));
    }
    if (il) {
      ProfScope ps(c, st, "paint", (catn[0] + catn[1]) * 16.0 + n3 * esz);
      CUDA_TRY(launch_paint<T>(cat4[0], catn[0], cat4[1], catn[1], stats, slot_r(ibase), N, p->box_lo, inv_h,
                               p->assign, pscr, c->nsm, st, 0.5));
    }
  }
  CUDA_TRY(cudaGetLastError());
  // forward plane transforms of painted and generated fields only over their occupied x planes
  // (library x pass backend; not in enqueued requests, which must not wait)
  XRange xr;
  const int fkind = fft_kind(c, N, p->precision, tn);
  if (!pd && !rq.full_planes && (fkind == 1 || fkind == 2 || fkind == 3)) {
    std::vector<const T *> ds = {slot_r(0)};
    if (il) ds.push_back(slot_r(ibase));
    if (cross) ds.push_back(slot_r(cbase));
    TRY(plane_range<T>(c, st, buf, ds, N, &xr));
    xr.rows = fkind == 1 || fkind == 3;
  }
  // field generation writes every value of the x planes [gx0, gx0 + gnp): the occupied range when
  // the x pass reads only the range's rows (the other planes are neither transformed nor read),
  // else every plane; and of those, the rows y in [gy0, gy0 + gny): the occupied rows when the
  // library's plane passes transform and read only those, else every row
  const int gx0 = (xr.np > 0 && xr.rows) ? xr.x0 : 0, gnp = (xr.np > 0 && xr.rows) ? xr.np : N;
  const int gy0 = (xr.ny > 0 && fkind == 3) ? xr.y0 : 0, gny = (xr.ny > 0 && fkind == 3) ? xr.ny : N;
  const long long gvals = (long long)gnp * gny * (N + kRowPad);
  static const char *kLosName[4] = {"yamamoto", "midpoint", "bisector", "midpoint_even"};
  const std::string los_name = kLosName[p->los];
  const std::string n_gen = "gen_fields_" + los_name, n_kc = "kcontract_" + los_name, n_xi = "xi_lag_" + los_name;
  const double cplx = 2.0 * esz * nhalf;  // one half-spectrum

  // field generation (streamed ranges generate their own fields below)
  if (!chunk) {
    ProfScope ps(c, st, n_gen.c_str(), (1.0 + nf) * gvals * esz * ((cross || il) ? 2.0 : 1.0));
    CUDA_TRY(launch(K.gen_fields, grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(0), slot_r(1),
                    slot_reals, N, p->box_lo[0], p->box_lo[1], p->box_lo[2], h, inv_r0, gx0, gnp, gy0, gny));
    if (cross) {   // tracer B's fields from its delta
      CUDA_TRY(launch(K.gen_fields, grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(cbase),
                      slot_r(cbase + 1), slot_reals, N, p->box_lo[0], p->box_lo[1], p->box_lo[2], h, inv_r0, gx0,
                      gnp, gy0, gny));
    }
    if (il) {   // the same fields on the shifted mesh, from its delta and node positions
      CUDA_TRY(launch(K.gen_fields, grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(ibase),
                      slot_r(ibase + 1), slot_reals, N, p->box_lo[0] + 0.5 * h, p->box_lo[1] + 0.5 * h,
                      p->box_lo[2] + 0.5 * h, h, inv_r0, gx0, gnp, gy0, gny));
    }
  }
  if (il) {
    // forward transforms of both sets (delta and the fields), then F <- (F + P G) / 2
    TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 0, 1 + nf, tn, &xr));
    TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, ibase, 1 + nf, tn, &xr));
    std::vector<T2> ph((size_t)N);
    for (int i = 0; i < N; ++i) {
      const int n = lab(i, N);
      const double a = -M_PI * n / N;
      ph[(size_t)i].x = n == -N / 2 ? (T)0 : (T)std::cos(a);
      ph[(size_t)i].y = n == -N / 2 ? (T)0 : (T)std::sin(a);
    }
    T2 *dph = nullptr;
    TRY(alloc((void **)&dph, sizeof(T2) * N));
    const void *src = ph.data();
    if (pd) {
      T2 *dst = (T2 *)(pd->stage + sizeof(double) * (size_t)nf + sizeof(T) * (size_t)N);
      std::copy(ph.begin(), ph.end(), dst);
      src = dst;
    }
    CUDA_TRY(cudaMemcpyAsync(dph, src, sizeof(T2) * N, cudaMemcpyHostToDevice, st));
    ProfScope ps(c, st, "interlace", (1.0 + nf) * 3.0 * cplx);
    launch_interlace<T, T2>(slot_c(0), slot_c(ibase), cslot, 1 + nf, N, dph, c->nsm, st);
  }

  const unsigned gk = grid_of((long long)N * N * (N / 2 + 1), c->nsm, tn.per_sm_k);
  const size_t smk = sums_smem(NL * nbk), smr = sums_smem(NL * nbr);
  const double tscale = h * inv_r0;

  double pk_scale = 1.0;
  if (cross) {
    // two tracers: A's delta and fields in slots [0, 1 + nf), B's in [cbase, cbase + 1 + nf)
    const bool bis = p->los == BYM_LOS_BISECTOR;
    const int f0 = bis ? 1 : 0, cnt = bis ? nf : 1 + nf;
    TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, f0, cnt, tn, &xr));
    TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, cbase + f0, cnt, tn, &xr));
    if (bis) {
      {
        ProfScope ps(c, st, "kcontract_bisector_cross", (2.0 * nf + (want_xi ? nlm : 0.0)) * cplx);
        CUDA_TRY(launch(kx, gk, 256, smk, st, (const T2 *)slot_c(1), (const T2 *)slot_c(cbase + 1), cslot, N,
                        (const int *)kg->lut, nbk, ksum, want_xi ? slot_c(xbase) : (T2 *)nullptr, cslot,
                        (const T *)invw, 0));
      }
      if (want_xi) {
        TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, xbase, nlm, tn));
        const int Lc = rg->full ? N : 2 * rg->jm + 1;
        ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nlm * esz);
        CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st,
                        (const T *)slot_r(xbase), slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum,
                        1.0 / ((double)N * N * N), tscale));
      }
    } else {
      if (p->los == BYM_LOS_YAMAMOTO && want_pk) {
        // the two endpoint lines of sight: F[Y delta_A] conj(D_B) + F[Y delta_B] conj(D_A), halved on the host
        pk_scale = 0.5;
        ProfScope ps(c, st, n_kc.c_str(), 2.0 * (nlm + 1.0) * 2.0 * esz * (double)kg->half_binned);
        CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(1), cslot, (const T2 *)slot_c(cbase), N,
                        (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)invw));
        CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(cbase + 1), cslot, (const T2 *)slot_c(0),
                        N, (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)invw));
      }
      if (is_midpoint(p) || want_xi) {
        // g = (g^AB + g^BA) / 2 (midpoint), the same product for the Yamamoto xi
        {
          ProfScope ps(c, st, "spec_mul_cross", (3.0 * nf + 2.0) * cplx);
          launch_spec_mul_cross<T, T2>(slot_c(1), slot_c(cbase + 1), cslot, nf, slot_c(0), slot_c(cbase), N, scale,
                                       invw, c->nsm * tn.per_sm_spec / 8, st);
        }
        TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1, nf, tn));
      }
      if (want_xi) {
        const int Lc = rg->full ? N : 2 * rg->jm + 1;
        ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nf * esz);
        CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(1),
                        slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
      }
      if (is_midpoint(p) && want_pk) {
        {
          ProfScope ps(c, st, "mid_combine", ((double)nf + nlm) * n3 * esz);
          CUDA_TRY(launch(K.mid_combine, grid_of((long long)N * N * N, c->nsm, tn.per_sm_comb), 256, 0, st,
                          (const T *)slot_r(1), slot_reals, slot_r(1 + nf), N, tscale));
        }
        TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 1 + nf, nlm, tn));
        ProfScope ps(c, st, n_kc.c_str(), nlm * 2.0 * esz * (double)kg->half_binned);
        CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(1 + nf), cslot, (const T2 *)slot_c(0), N,
                        (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)nullptr));
      }
    }
  } else if (p->los == BYM_LOS_YAMAMOTO) {
    if (!il) TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 0, 1 + nf, tn, &xr));
    if (want_pk) {
      ProfScope ps(c, st, n_kc.c_str(), (nlm + 1.0) * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(1), cslot, (const T2 *)slot_c(0), N,
                      (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)invw));
    }
    if (want_xi) {
      {
        ProfScope ps(c, st, "spec_mul", (2.0 * nf + 1.0) * cplx);
        launch_spec_mul<T, T2>(slot_c(1), cslot, nf, slot_c(0), N, scale, invw, c->nsm * tn.per_sm_spec / 8, st);
      }
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1, nf, tn));
      const int Lc = rg->full ? N : 2 * rg->jm + 1;
      ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nlm * esz);
      CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(1),
                      slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
    }
  } else if (chunk && is_midpoint(p)) {
    // delta's spectrum in slot 0, its real copy in slot 1 feeds gen_fields of every range
    CUDA_TRY(cudaMemcpyAsync(slot_r(1), slot_r(0), slot_bytes, cudaMemcpyDeviceToDevice, st));
    TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 0, 1, tn, &xr));
    for (size_t q = 0; q < CK->ranges.size(); ++q) {
      const int f0 = CK->ranges[q].first, nq = CK->ranges[q].second - f0;
      {
        ProfScope ps(c, st, n_gen.c_str(), (1.0 + nq) * gvals * esz);
        CUDA_TRY(launch(CK->gen[q], grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(1),
                        slot_r(2), slot_reals, N, p->box_lo[0], p->box_lo[1], p->box_lo[2], h, inv_r0, gx0, gnp, gy0, gny));
      }
      TRY((convolve_fields<T, T2>(c, st, p->precision, N, slots, slot_bytes, 2, nq, scale + f0, invw, tn, &xr)));
      if (want_xi) {
        const int Lc = rg->full ? N : 2 * rg->jm + 1;
        ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nq * esz);
        CUDA_TRY(launch(CK->xi[q], grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(2),
                        slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
      }
      if (want_pk) {
        ProfScope ps(c, st, "mid_combine", ((double)nq + (q ? 2.0 : 1.0) * nlm) * n3 * esz);
        CUDA_TRY(launch(CK->comb[q], grid_of((long long)N * N * N, c->nsm, tn.per_sm_comb), 256, 0, st,
                        (const T *)slot_r(2), slot_reals, slot_r(xbase), N, tscale));
      }
    }
    if (want_pk) {
      TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, xbase, nlm, tn));
      ProfScope ps(c, st, n_kc.c_str(), nlm * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(xbase), cslot, (const T2 *)slot_c(0), N,
                      (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)nullptr));
    }
  } else if (is_midpoint(p)) {
    if (il) {   // spectra ready (interlaced): the product and the inverse transforms
      {
        ProfScope ps(c, st, "spec_mul", (2.0 * nf + 1.0) * cplx);
        launch_spec_mul<T, T2>(slot_c(1), cslot, nf, slot_c(0), N, scale, invw, c->nsm * tn.per_sm_spec / 8, st);
      }
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1, nf, tn));
    } else {
      TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 0, 1, tn, &xr));
      TRY((convolve_fields<T, T2>(c, st, p->precision, N, slots, slot_bytes, 1, nf, scale, invw, tn, &xr)));
    }
    if (want_xi) {
      const int Lc = rg->full ? N : 2 * rg->jm + 1;
      ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nf * esz);
      CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(1),
                      slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
    }
    if (want_pk) {
      {
        ProfScope ps(c, st, "mid_combine", ((double)nf + nlm) * n3 * esz);
        CUDA_TRY(launch(K.mid_combine, grid_of((long long)N * N * N, c->nsm, tn.per_sm_comb), 256, 0, st,
                        (const T *)slot_r(1), slot_reals, slot_r(1 + nf), N, tscale));
      }
      TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 1 + nf, nlm, tn));
      ProfScope ps(c, st, n_kc.c_str(), nlm * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(1 + nf), cslot, (const T2 *)slot_c(0), N,
                      (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)nullptr));
    }
  } else if (bis_blocks) {
    // blocks A (slots 1..) and B (slots 1 + chunk..); every block pair a <= b adds its
    // share of the bilinear sum: block a transformed once, every later block once per a
    const int nb = (int)CK->ranges.size();
    auto make_block = [&](int q, int base) -> int {
      const int q0 = CK->ranges[q].first, nq = CK->ranges[q].second - q0;
      {
        ProfScope ps(c, st, n_gen.c_str(), (1.0 + nq) * gvals * esz);
        CUDA_TRY(launch(CK->gen[q], grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(0),
                        slot_r(base), slot_reals, N, p->box_lo[0], p->box_lo[1], p->box_lo[2], h, inv_r0, gx0, gnp, gy0, gny));
      }
      return fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, base, nq, tn, &xr);
    };
    T2 *xout = want_xi ? slot_c(xbase) : nullptr;
    int accumulate = 0;
    for (int a = 0; a < nb; ++a) {
      TRY(make_block(a, 1));
      for (int b = a; b < nb; ++b) {
        if (b > a) TRY(make_block(b, 1 + chunk));
        const double nfa = CK->ranges[a].second - CK->ranges[a].first;
        const double nfb = b > a ? CK->ranges[b].second - CK->ranges[b].first : 0.0;
        ProfScope ps(c, st, "kcontract_bisector_pair", (nfa + nfb + (want_xi ? 2.0 * nlm : 0.0)) * cplx);
        CUDA_TRY(launch(CK->pair[(size_t)a * nb + b], gk, 256, smk, st, (const T2 *)slot_c(1),
                        (const T2 *)slot_c(b > a ? 1 + chunk : 1), cslot, N, (const int *)kg->lut, nbk, ksum, xout,
                        cslot, (const T *)invw, accumulate));
        accumulate = 1;
      }
    }
    if (want_xi) {
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, xbase, nlm, tn));
      const int Lc = rg->full ? N : 2 * rg->jm + 1;
      ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nlm * esz);
      CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st,
                      (const T *)slot_r(xbase), slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum,
                      1.0 / ((double)N * N * N), tscale));
    }
  } else {
    if (!il) TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, 1, nf, tn, &xr));
    if (want_xi) {
      {
        ProfScope ps(c, st, "kcontract_bisector_x", ((double)nf + nlm) * cplx);
        CUDA_TRY(launch(K.kcontract_x, gk, 256, smk, st, (const T2 *)slot_c(1), cslot, (const T2 *)slot_c(0), N,
                        (const int *)kg->lut, nbk, ksum, slot_c(1 + nf), cslot, (const T *)invw));
      }
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1 + nf, nlm, tn));
      const int Lc = rg->full ? N : 2 * rg->jm + 1;
      ProfScope ps(c, st, n_xi.c_str(), (double)Lc * Lc * Lc * nlm * esz);
      CUDA_TRY(launch(K.xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st,
                      (const T *)slot_r(1 + nf), slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum,
                      1.0 / ((double)N * N * N), tscale));
    } else {
      ProfScope ps(c, st, n_kc.c_str(), (double)nf * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(K.kcontract, gk, 256, smk, st, (const T2 *)slot_c(1), cslot, (const T2 *)slot_c(0), N,
                      (const int *)kg->lut, nbk, ksum, (T2 *)nullptr, 0LL, (const T *)invw));
    }
  }
  CUDA_TRY(cudaGetLastError());

  // results
  if (pd) {
    double *hs = pd->host;
    CUDA_TRY(cudaMemcpyAsync(hs, stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hs + 8, ksum, sizeof(double) * NL * nbk, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hs + 8 + NL * nbk, rsum, sizeof(double) * NL * nbr, cudaMemcpyDeviceToHost, st));
    pd->kg = kg;
    pd->rg = rg;
    pd->NL = NL;
    pd->nbk = nbk;
    pd->nbr = nbr;
    pd->h = h;
    return BYM_OK;
  }
  std::vector<double> hstats(16), hk((size_t)NL * nbk), hr((size_t)NL * nbr);
  CUDA_TRY(cudaMemcpyAsync(hstats.data(), stats, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hk.data(), ksum, hk.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hr.data(), rsum, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  prof_collect(c);
  return finish_results(c, rq, hstats.data(), hk.data(), hr.data(), kg, rg, NL, nbk, nbr, h, cross, pk_scale);
#undef TRY
#undef CUDA_TRY
}

// Odd multipoles l = 1, 3, .., ell_max of a cross spectrum (Yamamoto or bisector; ell_max odd):
// the relabelled first-galaxy terms keep a factor (-1)^l, so the Yamamoto form is
// [Q^AB - Q^BA] / 2 with Q^XY = F[Y delta_Y] conj(D_X), and the bisector sum of eq.
// bisector-pk-fft contributes its part odd in k, sum c_ij Im(conj F^A_i F^B_j); P_l is the
// imaginary part of the shell mean, xi_l the (real) lag sum.  Tracer A: slot 0 and its fields
// from slot 1, the bisector X fields (xi) after them, tracer B's delta and fields last.
template <typename T, typename T2>
static int run_odd(bym_ctx *c, const Request &rq, cudaStream_t st) {
  const bym_params *p = rq.p;
  const int N = p->n_mesh;
  const bool want_pk = rq.kb != nullptr, want_xi = rq.rb != nullptr, bis = p->los == BYM_LOS_BISECTOR;
  std::string jerr;
  auto os = get_odd_kernels(JitKey{p->los, p->ell_max, order_key(p), p->precision}, jerr);
  if (!os) return fail(c, BYM_E_CUDA, jerr);
  auto ks = get_kernels(JitKey{p->los, p->ell_max - 1, order_key(p), p->precision}, jerr);   // bin geometry
  if (!ks) return fail(c, BYM_E_CUDA, jerr);
  const Tune &tn = tune_for(c, N, p->precision, p->los);
  const int nf = (int)os->fields.size(), nlm = os->n_lm, NL = os->n_ell;
  const long long slot_reals = (long long)N * N * (N + kRowPad), cslot = slot_reals / 2;
  const size_t slot_bytes = (size_t)slot_reals * sizeof(T);
  const double h = p->box_len / N, inv_h = N / p->box_len, inv_r0 = 1.0 / p->box_len;
  const bool mid = p->los == BYM_LOS_MIDPOINT;
  const int nextra = (bis && want_xi) || (mid && want_pk) ? nlm : 0;   // bisector X (xi) or midpoint H (P)
  const int xbase = 1 + nf, cbase = xbase + nextra, nslots = cbase + 1 + nf;
  const double tscale = h * inv_r0;
  const int64_t ncat = rq.gal->n + rq.gal_b->n + (rq.ran ? rq.ran->n : 0) + (rq.ran_b ? rq.ran_b->n : 0);
  const bool cats_dev = rq.gal->on_device && rq.gal_b->on_device && (!rq.ran || rq.ran->on_device) &&
                        (!rq.ran_b || rq.ran_b->on_device);
  if (c->budget && (size_t)nslots * slot_bytes + (cats_dev ? 0 : (size_t)ncat * 20) > c->budget)
    return fail(c, BYM_E_NOMEM, "request exceeds the context's HBM budget");

  Geom *kg = nullptr, *rg = nullptr;
  int rc;
  if (want_pk && (rc = get_geom(c, *ks, N, p->box_len, rq.kb, 'k', st, &kg))) return rc;
  if (want_xi && (rc = get_geom(c, *ks, N, p->box_len, rq.rb, 'r', st, &rg))) return rc;
  if (!kg && bis && (rc = get_null_kgeom(c, N, &kg))) return rc;

  DevBufs buf(st);
  auto alloc = [&](void **ptr, size_t bytes) -> int {
    if (buf.alloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, BYM_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return BYM_OK;
  };
#define TRY(x)                  \
  do {                          \
    int rc_ = (x);              \
    if (rc_) return rc_;        \
  } while (0)
#define CUDA_TRY(x)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return fail(c, BYM_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

  const bym_catalog *cats[4] = {rq.gal, rq.ran, rq.gal_b, rq.ran_b};
  const float4 *cat4[4] = {nullptr, nullptr, nullptr, nullptr};
  const float *catnb[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int w = 0; w < 4; ++w) {
    const bym_catalog *cat = cats[w];
    if (!cat || cat->n <= 0) continue;
    if (cat->on_device) {
      cat4[w] = (const float4 *)cat->xyzw;
      catnb[w] = cat->nbar;
      continue;
    }
    void *d4 = nullptr;
    TRY(alloc(&d4, (size_t)cat->n * 16));
    CUDA_TRY(cudaMemcpyAsync(d4, cat->xyzw, (size_t)cat->n * 16, cudaMemcpyHostToDevice, st));
    cat4[w] = (const float4 *)d4;
    if (cat->nbar) {
      void *dn = nullptr;
      TRY(alloc(&dn, (size_t)cat->n * 4));
      CUDA_TRY(cudaMemcpyAsync(dn, cat->nbar, (size_t)cat->n * 4, cudaMemcpyHostToDevice, st));
      catnb[w] = (const float *)dn;
    }
  }
  double *stats = nullptr, *ksum = nullptr, *rsum = nullptr, *scale = nullptr;
  T *invw = nullptr;
  const int nbk = want_pk ? rq.kb->nbins : 1, nbr = want_xi ? rq.rb->nbins : 1;
  TRY(alloc((void **)&stats, 16 * sizeof(double)));
  TRY(alloc((void **)&ksum, sizeof(double) * sums_doubles(NL * nbk, c->nsm, std::max(tn.per_sm_k, 1))));
  TRY(alloc((void **)&rsum, sizeof(double) * sums_doubles(NL * nbr, c->nsm, 4)));
  CUDA_TRY(cudaMemsetAsync(stats, 0, 16 * sizeof(double), st));
  CUDA_TRY(cudaMemsetAsync(ksum, 0, sizeof(double) * (NL * nbk + 1), st));
  CUDA_TRY(cudaMemsetAsync(rsum, 0, sizeof(double) * (NL * nbr + 1), st));
  if (p->compensate) {
    std::vector<T> w(N);
    for (int i = 0; i < N; ++i) {
      const double x = M_PI * lab(i, N) / N;
      const double sn = x == 0.0 ? 1.0 : std::sin(x) / x;
      w[i] = (T)(1.0 / std::pow(sn, p->assign));
    }
    TRY(alloc((void **)&invw, sizeof(T) * N));
    CUDA_TRY(cudaMemcpyAsync(invw, w.data(), sizeof(T) * N, cudaMemcpyHostToDevice, st));
  }
  // midpoint: g = [-g^AB + g^BA] / 2 with the (-1)^J of eq. g-JM-form, from the product
  // [-F^A conj(D_B) + F^B conj(D_A)] s / 2 with s = -(-1)^J / N^3
  std::vector<double> sc((size_t)nf, 1.0 / ((double)N * N * N));
  if (mid)
    for (int i = 0; i < nf; ++i) sc[(size_t)i] *= (os->fields[(size_t)i].J % 2) ? 1.0 : -1.0;
  TRY(alloc((void **)&scale, sizeof(double) * nf));
  CUDA_TRY(cudaMemcpyAsync(scale, sc.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, st));

  T *slots = nullptr;
  TRY(alloc((void **)&slots, (size_t)nslots * slot_bytes));
  auto slot_r = [&](int i) { return slots + (long long)i * slot_reals; };
  auto slot_c = [&](int i) { return (T2 *)(slots + (long long)i * slot_reals); };
  const double esz = (double)sizeof(T), n3 = (double)N * N * N, cplx = 2.0 * esz * N * N * (N / 2 + 1);
  double *npart = nullptr;
  TRY(alloc((void **)&npart, norm_scratch_bytes(c->nsm)));
  long long catn[4];
  for (int w = 0; w < 4; ++w) catn[w] = cat4[w] ? cats[w]->n : 0;
  for (int w = 0; w < 4; ++w)
    if (cat4[w]) {
      ProfScope ps(c, st, "norm_reduce", catn[w] * ((w & 1) ? 20.0 : 16.0));
      launch_norm_reduce(cat4[w], catnb[w], catn[w], w & 1, p->box_lo, inv_h, N, stats + 8 * (w >> 1), npart, c->nsm,
                         st, p->precision);
    }
  {
    void *pscr = nullptr;
    TRY(alloc(&pscr, paint_scratch_bytes(N, std::max(catn[0] + catn[1], catn[2] + catn[3]))));
    for (int t = 0; t < 2; ++t) {
      const int w = 2 * t;
      ProfScope ps(c, st, "paint", (catn[w] + catn[w + 1]) * 16.0 + n3 * esz);
      CUDA_TRY(launch_paint<T>(cat4[w], catn[w], cat4[w + 1], catn[w + 1], stats + 8 * t, slot_r(t ? cbase : 0), N,
                               p->box_lo, inv_h, p->assign, pscr, c->nsm, st));
    }
  }
  CUDA_TRY(cudaGetLastError());
  XRange xr;   // forward plane transforms over the occupied x planes (plane-transform backends)
  const int fkind = fft_kind(c, N, p->precision, tn);
  if (fkind == 1 || fkind == 2 || fkind == 3) {
    TRY(plane_range<T>(c, st, buf, {slot_r(0), slot_r(cbase)}, N, &xr));
    xr.rows = fkind == 1 || fkind == 3;
  }
  {
    // every value of the rows [gy0, gy0 + gny) of the planes [gx0, gx0 + gnp) of every field (see run_typed)
    const int gx0 = (xr.np > 0 && xr.rows) ? xr.x0 : 0, gnp = (xr.np > 0 && xr.rows) ? xr.np : N;
    const int gy0 = (xr.ny > 0 && fkind == 3) ? xr.y0 : 0, gny = (xr.ny > 0 && fkind == 3) ? xr.ny : N;
    const long long gvals = (long long)gnp * gny * (N + kRowPad);
    ProfScope ps(c, st, "gen_fields_odd", 2.0 * (1.0 + nf) * gvals * esz);
    for (int base : {0, cbase})
      CUDA_TRY(launch(os->gen_fields, grid_of(gvals, c->nsm, tn.per_sm_gen), 256, 0, st, (const T *)slot_r(base),
                      slot_r(base + 1), slot_reals, N, p->box_lo[0], p->box_lo[1], p->box_lo[2], h, inv_r0, gx0,
                      gnp, gy0, gny));
  }
  const int f0 = bis ? 1 : 0, cnt = bis ? nf : 1 + nf;
  TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, f0, cnt, tn, &xr));
  TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, cbase + f0, cnt, tn, &xr));
  const unsigned gk = grid_of((long long)N * N * (N / 2 + 1), c->nsm, tn.per_sm_k);
  const size_t smk = sums_smem(NL * nbk), smr = sums_smem(NL * nbr);
  const int Lc = want_xi ? (rg->full ? N : 2 * rg->jm + 1) : 0;
  double pk_scale = 1.0;
  if (bis) {
    {
      ProfScope ps(c, st, "kcontract_bisector_cross_odd", (2.0 * nf + (want_xi ? nlm : 0.0)) * cplx);
      CUDA_TRY(launch(os->kcontract, gk, 256, smk, st, (const T2 *)slot_c(1), (const T2 *)slot_c(cbase + 1), cslot,
                      N, (const int *)kg->lut, nbk, ksum, want_xi ? slot_c(xbase) : (T2 *)nullptr, cslot,
                      (const T *)invw));
    }
    if (want_xi) {
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, xbase, nlm, tn));
      ProfScope ps(c, st, "xi_lag_odd", (double)Lc * Lc * Lc * nlm * esz);
      CUDA_TRY(launch(os->xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st,
                      (const T *)slot_r(xbase), slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum,
                      1.0 / ((double)N * N * N), tscale));
    }
  } else if (mid) {
    {
      ProfScope ps(c, st, "spec_mul_cross", (3.0 * nf + 2.0) * cplx);
      launch_spec_mul_cross<T, T2>(slot_c(1), slot_c(cbase + 1), cslot, nf, slot_c(0), slot_c(cbase), N, scale, invw,
                                   c->nsm * tn.per_sm_spec / 8, st, -1.0);
    }
    TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1, nf, tn));
    if (want_xi) {
      ProfScope ps(c, st, "xi_lag_odd", (double)Lc * Lc * Lc * nf * esz);
      CUDA_TRY(launch(os->xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(1),
                      slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
    }
    if (want_pk) {
      {
        ProfScope ps(c, st, "mid_combine_odd", ((double)nf + nlm) * n3 * esz);
        CUDA_TRY(launch(os->mid_combine, grid_of((long long)N * N * N, c->nsm, tn.per_sm_comb), 256, 0, st,
                        (const T *)slot_r(1), slot_reals, slot_r(xbase), N, tscale));
      }
      TRY(fft_slots(c, st, p->precision, 0, N, slots, slot_bytes, xbase, nlm, tn));
      ProfScope ps(c, st, "kcontract_midpoint_odd", nlm * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(os->kcontract, gk, 256, smk, st, (const T2 *)slot_c(xbase), cslot, N, (const int *)kg->lut, nbk,
                      ksum));
    }
  } else {
    if (want_pk) {
      // [Q^AB - Q^BA], halved on the host: F^B with D_A (+), F^A with D_B (-)
      pk_scale = 0.5;
      ProfScope ps(c, st, "kcontract_yamamoto_odd", 2.0 * (nlm + 1.0) * 2.0 * esz * (double)kg->half_binned);
      CUDA_TRY(launch(os->kcontract, gk, 256, smk, st, (const T2 *)slot_c(cbase + 1), cslot, (const T2 *)slot_c(0),
                      N, (const int *)kg->lut, nbk, ksum, (const T *)invw, (T)1));
      CUDA_TRY(launch(os->kcontract, gk, 256, smk, st, (const T2 *)slot_c(1), cslot, (const T2 *)slot_c(cbase), N,
                      (const int *)kg->lut, nbk, ksum, (const T *)invw, (T)-1));
    }
    if (want_xi) {
      {
        ProfScope ps(c, st, "spec_mul_cross", (3.0 * nf + 2.0) * cplx);
        launch_spec_mul_cross<T, T2>(slot_c(1), slot_c(cbase + 1), cslot, nf, slot_c(0), slot_c(cbase), N, scale,
                                     invw, c->nsm * tn.per_sm_spec / 8, st, -1.0);
      }
      TRY(fft_slots(c, st, p->precision, 1, N, slots, slot_bytes, 1, nf, tn));
      ProfScope ps(c, st, "xi_lag_odd", (double)Lc * Lc * Lc * nf * esz);
      CUDA_TRY(launch(os->xi_lag, grid_of((long long)Lc * Lc * Lc, c->nsm, 4), 256, smr, st, (const T *)slot_r(1),
                      slot_reals, N, rg->jm, rg->full, (const int *)rg->lut, nbr, rsum, 1.0, tscale));
    }
  }
  CUDA_TRY(cudaGetLastError());
  std::vector<double> hstats(16), hk((size_t)NL * nbk), hr((size_t)NL * nbr);
  CUDA_TRY(cudaMemcpyAsync(hstats.data(), stats, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hk.data(), ksum, hk.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hr.data(), rsum, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  prof_collect(c);
  return finish_results(c, rq, hstats.data(), hk.data(), hr.data(), kg, rg, NL, nbk, nbr, h, true, pk_scale);
#undef TRY
#undef CUDA_TRY
}

// norm 2 (Sec. 2.2: the Landy-Szalay form of the catalog pair counts): P with the
// FKP normalisation; xi_ell(r_b) = S_ell[delta](b) / (alpha_r^2 S_0[n_r](b)), both raw
// bin sums of the same mesh estimator; the random-random sum is the ell = 0 one, where
// the line of sight drops out, computed with the Yamamoto form.  Bins without random
// pairs give 0.
static int run_rr_normalised(bym_ctx *c, const Request &rq, cudaStream_t st) {
  const bool f64 = rq.p->precision == 64;
  double alpha = 0.0;
  Request main = rq;
  main.alpha = &alpha;
  int rc = f64 ? run_typed<double, double2>(c, main, st) : run_typed<float, float2>(c, main, st);
  if (rc) return rc;
  bym_params pr = *rq.p;
  pr.los = BYM_LOS_YAMAMOTO;
  pr.ell_max = 0;
  pr.order = 0;
  pr.norm = 0;
  const int nbr = rq.rb->nbins, NL = rq.p->ell_max / 2 + 1;
  std::vector<double> rr((size_t)nbr);
  Request rrq{rq.ran, nullptr, &pr, nullptr, rq.rb, nullptr, nullptr, nullptr, rr.data(), nullptr, nullptr};
  rc = f64 ? run_typed<double, double2>(c, rrq, st) : run_typed<float, float2>(c, rrq, st);
  if (rc) return rc;
  for (int b = 0; b < nbr; ++b) {
    const double den = alpha * alpha * rr[b];
    for (int l = 0; l < NL; ++l) rq.xi[l * nbr + b] = den != 0.0 ? rq.xi[l * nbr + b] / den : 0.0;
  }
  return BYM_OK;
}

int bym::run_request(bym_ctx *c, const Request &rq, cudaStream_t st) {
  if (!c) return BYM_E_INVAL;
  if (rq.odd) {   // odd multipoles: ell_max odd; the rest is checked as for ell_max - 1
    const bym_params *p = rq.p;
    if (!p || !rq.gal_b) return fail(c, BYM_E_INVAL, "odd multipoles: params and two tracers are required");
    if (p->ell_max < 1 || p->ell_max > 7 || p->ell_max % 2 == 0)
      return fail(c, BYM_E_UNSUPPORTED, "odd multipoles: ell_max must be odd, 1..7");
    if (p->los == BYM_LOS_MIDPOINT_EVEN)
      return fail(c, BYM_E_UNSUPPORTED, "odd multipoles: the parity-even midpoint form is even-ell only");
    if (p->norm == 2 || p->interlace || (c->field_chunk > 0 && p->los != BYM_LOS_YAMAMOTO))
      return fail(c, BYM_E_UNSUPPORTED, "odd multipoles: no norm 2, no interlacing, no field ranges or blocks");
    bym_params pe = *p;
    pe.ell_max = p->ell_max - 1;
    int rc = validate(c, rq.gal, rq.ran, &pe, rq.kb, rq.rb);
    if (!rc) rc = validate(c, rq.gal_b, rq.ran_b, &pe, rq.kb, rq.rb);
    if (rc) return rc;
    if ((rq.kb && !rq.pk) || (rq.rb && !rq.xi) || (!rq.kb && !rq.rb))
      return fail(c, BYM_E_INVAL, "missing output array");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
    if (!st) st = c->stream;
    try {
      return p->precision == 64 ? run_odd<double, double2>(c, rq, st) : run_odd<float, float2>(c, rq, st);
    } catch (const std::exception &e) {
      return fail(c, BYM_E_CUDA, std::string("internal error: ") + e.what());
    }
  }
  int rc = validate(c, rq.gal, rq.ran, rq.p, rq.kb, rq.rb);
  if (rc) return rc;
  if (rq.gal_b && (rc = validate(c, rq.gal_b, rq.ran_b, rq.p, rq.kb, rq.rb))) return rc;
  if (rq.gal_b && (rq.p->norm == 2 || rq.p->interlace))
    return fail(c, BYM_E_UNSUPPORTED, "cross spectra: norm 2 and interlacing are not available");
  if ((rq.kb && !rq.pk) || (rq.rb && !rq.xi) || (!rq.kb && !rq.rb))
    return fail(c, BYM_E_INVAL, "missing output array");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  if (!st) st = c->stream;
  try {
    if (rq.p->norm == 2 && rq.rb) return run_rr_normalised(c, rq, st);
    if (rq.p->precision == 64) return run_typed<double, double2>(c, rq, st);
    return run_typed<float, float2>(c, rq, st);
  } catch (const std::exception &e) {
    return fail(c, BYM_E_CUDA, std::string("internal error: ") + e.what());
  }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *bym_version(void) { return "bym 0.1 (sm_103a)"; }

int bym_create(bym_ctx **out, int device, size_t hbm_budget_bytes) {
  if (!out) return BYM_E_INVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BYM_E_CUDA;
  }
  auto *c = new bym_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreate(&c->stream) != cudaSuccess) {   // a blocking stream: orders after legacy-stream work
    cudaGetLastError();
    delete c;
    return BYM_E_CUDA;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  *out = c;
  return BYM_OK;
}

void bym_destroy(bym_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  shutdown_serving(c);
  for (auto &kv : c->plans) cufftDestroy(kv.second);
  for (auto &p : c->prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->fft_work) cudaFreeAsync(c->fft_work, c->stream);
  cudaStreamSynchronize(c->stream);
  for (auto *m : {&c->kgeo, &c->rgeo})
    for (auto &kv : *m)
      if (kv.second.lut) cudaFree(kv.second.lut);
  cudaStreamDestroy(c->stream);
  delete c;
}

const char *bym_last_error(const bym_ctx *c) { return c ? c->err.c_str() : "no context"; }

int bym_footprint(const bym_params *p, int64_t n_gal, int64_t n_ran, int want_pk, int want_xi, size_t *bytes) {
  if (!p || !bytes) return BYM_E_INVAL;
  int rc = validate_params(nullptr, p);
  if (rc) return rc;
  *bytes = footprint_bytes(p, n_gal, n_ran, want_pk != 0, want_xi != 0, false);
  return BYM_OK;
}

int bym_pk_multipoles(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                      const bym_bins *kbins, double *pk, double *k_mean, int64_t *n_modes, void *stream) {
  if (!c) return BYM_E_INVAL;
  if (!kbins) return fail(c, BYM_E_INVAL, "kbins is NULL");
  std::lock_guard<std::mutex> lock(c->mu);
  Request rq{gal, ran, p, kbins, nullptr, pk, k_mean, n_modes, nullptr, nullptr, nullptr};
  return run_request(c, rq, (cudaStream_t)stream);
}

int bym_xi_multipoles(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                      const bym_bins *rbins, double *xi, double *r_mean, int64_t *n_cells, void *stream) {
  if (!c) return BYM_E_INVAL;
  if (!rbins) return fail(c, BYM_E_INVAL, "rbins is NULL");
  std::lock_guard<std::mutex> lock(c->mu);
  Request rq{gal, ran, p, nullptr, rbins, nullptr, nullptr, nullptr, xi, r_mean, n_cells};
  return run_request(c, rq, (cudaStream_t)stream);
}

int bym_pk_xi_multipoles(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                         const bym_bins *kbins, const bym_bins *rbins, double *pk, double *k_mean, int64_t *n_modes,
                         double *xi, double *r_mean, int64_t *n_cells, void *stream) {
  if (!c) return BYM_E_INVAL;
  if (!kbins || !rbins) return fail(c, BYM_E_INVAL, "kbins and rbins are required");
  std::lock_guard<std::mutex> lock(c->mu);
  Request rq{gal, ran, p, kbins, rbins, pk, k_mean, n_modes, xi, r_mean, n_cells};
  return run_request(c, rq, (cudaStream_t)stream);
}

int bym_pk_xi_cross(bym_ctx *c, const bym_catalog *gal_a, const bym_catalog *ran_a, const bym_catalog *gal_b,
                    const bym_catalog *ran_b, const bym_params *p, const bym_bins *kbins, const bym_bins *rbins,
                    double *pk, double *k_mean, int64_t *n_modes, double *xi, double *r_mean, int64_t *n_cells,
                    void *stream) {
  if (!c) return BYM_E_INVAL;
  if (!gal_b) return fail(c, BYM_E_INVAL, "gal_b is NULL");
  if (!kbins && !rbins) return fail(c, BYM_E_INVAL, "kbins or rbins is required");
  std::lock_guard<std::mutex> lock(c->mu);
  Request rq{gal_a, ran_a, p, kbins, rbins, pk, k_mean, n_modes, xi, r_mean, n_cells};
  rq.gal_b = gal_b;
  rq.ran_b = ran_b;
  return run_request(c, rq, (cudaStream_t)stream);
}

int bym_pk_xi_cross_odd(bym_ctx *c, const bym_catalog *gal_a, const bym_catalog *ran_a, const bym_catalog *gal_b,
                        const bym_catalog *ran_b, const bym_params *p, const bym_bins *kbins, const bym_bins *rbins,
                        double *pk, double *k_mean, int64_t *n_modes, double *xi, double *r_mean, int64_t *n_cells,
                        void *stream) {
  if (!c) return BYM_E_INVAL;
  if (!gal_b) return fail(c, BYM_E_INVAL, "gal_b is NULL");
  if (!kbins && !rbins) return fail(c, BYM_E_INVAL, "kbins or rbins is required");
  std::lock_guard<std::mutex> lock(c->mu);
  Request rq{gal_a, ran_a, p, kbins, rbins, pk, k_mean, n_modes, xi, r_mean, n_cells};
  rq.gal_b = gal_b;
  rq.ran_b = ran_b;
  rq.odd = true;
  return run_request(c, rq, (cudaStream_t)stream);
}

int bym_set_fft_backend(bym_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 6) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  c->fft_mode = mode;
  c->graph_warm.clear();   // other plans and kernels: warm again before the next captured batch
  return BYM_OK;
}

// A batch captured as one CUDA graph.  Every request (and, for norm 2, its
// random-random pass) is enqueued on one stream under capture; a launch runs the
// graph and normalises the results on the host.  Before the capture host catalogs
// are copied to the device and one request of every distinct shape not yet warmed on
// the context runs uncaptured, so that the captured requests find their kernels, bin
// tables, FFT plans and work area ready.
struct bym_batch {
  struct Item {
    bym_catalog gal{}, ran{};
    bym_params p{}, prr{};
    Request rq{}, rrq{};
    std::vector<double> rr;
    double alpha = 0.0;
    Pending pd, pdr;
    bool ok = false;
    int status = BYM_OK;          // validation / warm-up outcome
    int branch = 0;               // graph branch (engine and stream) that runs it
  };
  bym_ctx *c = nullptr;
  std::vector<bym_ctx *> eng;     // one engine per branch: its own FFT plans, work area, bin tables
  std::vector<cudaStream_t> bst;  // one stream per branch, forked from and joined to cs in the capture
  std::vector<cudaEvent_t> ev;
  std::vector<Item> it;
  std::vector<void *> dev;        // device copies of host catalogs
  char *pinned = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  ~bym_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t q : bst) cudaStreamDestroy(q);
    for (bym_ctx *e : eng) bym_destroy(e);
    if (cs) cudaStreamDestroy(cs);
    if (pinned) cudaFreeHost(pinned);
    for (void *q : dev) cudaFree(q);
    if (c) cudaDeviceGraphMemTrim(c->device);
  }
};

static int batch_create(bym_ctx *c, int n, const bym_request *reqs, const bym_result *outs, int n_streams,
                        std::unique_ptr<bym_batch> &out) {
  auto B = std::make_unique<bym_batch>();
  B->c = c;
  B->it.resize((size_t)n);
  cudaStream_t st = c->stream;   // warm-up runs here; the capture runs on its own non-blocking stream
  for (int i = 0; i < n; ++i) {
    auto &m = B->it[(size_t)i];
    m.gal = reqs[i].gal;
    m.ran = reqs[i].ran;
    m.p = reqs[i].params;
    const bym_bins *kb = reqs[i].kbins.nbins > 0 ? &reqs[i].kbins : nullptr;
    const bym_bins *rb = reqs[i].rbins.nbins > 0 ? &reqs[i].rbins : nullptr;
    const bym_catalog *ranp = m.ran.n > 0 ? &m.ran : nullptr;
    int rc = validate(c, &m.gal, ranp, &m.p, kb, rb);
    if (!rc && ((kb && !outs[i].pk) || (rb && !outs[i].xi) || (!kb && !rb)))
      rc = fail(c, BYM_E_INVAL, "missing output array");
    if (rc) {
      m.status = rc;
      continue;
    }
    for (bym_catalog *cat : {&m.gal, &m.ran}) {
      if (cat->n <= 0 || cat->on_device) continue;
      void *d4 = nullptr, *dn = nullptr;
      if (cudaMalloc(&d4, (size_t)cat->n * 16) != cudaSuccess ||
          (cat->nbar && cudaMalloc(&dn, (size_t)cat->n * 4) != cudaSuccess)) {
        cudaGetLastError();
        if (d4) cudaFree(d4);
        return fail(c, BYM_E_NOMEM, "batch: device copy of a catalog failed");
      }
      B->dev.push_back(d4);
      cudaMemcpy(d4, cat->xyzw, (size_t)cat->n * 16, cudaMemcpyHostToDevice);
      if (dn) {
        B->dev.push_back(dn);
        cudaMemcpy(dn, cat->nbar, (size_t)cat->n * 4, cudaMemcpyHostToDevice);
      }
      cat->xyzw = (const float *)d4;
      cat->nbar = (const float *)dn;
      cat->on_device = 1;
    }
    ranp = m.ran.n > 0 ? &m.ran : nullptr;
    m.rq = Request{&m.gal, ranp, &m.p, kb, rb, outs[i].pk, outs[i].k_mean, outs[i].n_modes,
                   outs[i].xi, outs[i].r_mean, outs[i].n_cells};
    m.rq.alpha = &m.alpha;
    if (m.p.norm == 2 && rb) {   // the random-random pass: Yamamoto, ell = 0, raw, xi only, on the randoms
      m.prr = m.p;
      m.prr.los = BYM_LOS_YAMAMOTO;
      m.prr.ell_max = 0;
      m.prr.order = 0;
      m.prr.norm = 0;
      m.rr.assign((size_t)rb->nbins, 0.0);
      m.rrq = Request{&m.ran, nullptr, &m.prr, nullptr, rb, nullptr, nullptr, nullptr, m.rr.data(), nullptr, nullptr};
    }
    m.ok = true;
  }
  // branches: engines created like serving slots, with this context's settings; the
  // requests go to the least loaded branch, largest first
  int n_ok = 0;
  for (auto &m : B->it) n_ok += m.ok ? 1 : 0;
  const int nb = std::max(1, std::min(n_streams > 0 ? n_streams : 4, std::max(n_ok, 1)));
  for (int b = 0; b < nb; ++b) {
    bym_ctx *e = nullptr;
    if (bym_create(&e, c->device, 0) != BYM_OK) return fail(c, BYM_E_CUDA, "batch: could not create a branch");
    e->tune = c->tune;
    e->fft_mode = c->fft_mode;
    e->field_chunk = c->field_chunk;
    B->eng.push_back(e);
  }
  {
    std::vector<std::pair<double, int>> order;
    for (int i = 0; i < n; ++i)
      if (B->it[(size_t)i].ok) {
        const bym_params &p = B->it[(size_t)i].p;
        order.push_back({std::pow((double)p.n_mesh, 3) * (2.0 + n_fields(&p)), i});
      }
    std::sort(order.rbegin(), order.rend());
    std::vector<double> load((size_t)nb, 0.0);
    for (auto &oi : order) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      B->it[(size_t)oi.second].branch = b;
      load[(size_t)b] += oi.first;
    }
  }
  auto shape_key = [](const Request &rq) {
    std::ostringstream o;
    const bym_params *p = rq.p;
    o << p->n_mesh << ':' << p->precision << ':' << p->los << ':' << p->ell_max << ':' << p->order << ':'
      << p->compensate << ':' << p->box_len << ':' << (rq.ran != nullptr) << ':';
    for (const bym_bins *b : {rq.kb, rq.rb}) {
      o << '|';
      if (b) o.write((const char *)b->edges, sizeof(double) * (b->nbins + 1));
    }
    return o.str();
  };
  for (auto &m : B->it) {        // an item whose warm-up fails reports it and leaves the batch
    if (!m.ok) continue;
    bym_ctx *e = B->eng[(size_t)m.branch];
    for (Request *rq : {&m.rq, m.rr.empty() ? nullptr : &m.rrq}) {
      if (!m.ok || !rq) continue;
      const std::string key = shape_key(*rq);
      if (e->graph_warm.count(key)) continue;
      const int NL = rq->p->ell_max / 2 + 1, nbk = rq->kb ? rq->kb->nbins : 0, nbr = rq->rb ? rq->rb->nbins : 0;
      std::vector<double> a((size_t)NL * nbk + 1), b((size_t)nbk + 1), d((size_t)NL * nbr + 1), f2((size_t)nbr + 1);
      std::vector<int64_t> f((size_t)nbk + 1), g((size_t)nbr + 1);
      Request w{rq->gal, rq->ran, rq->p, rq->kb, rq->rb, a.data(), b.data(), f.data(), d.data(), f2.data(), g.data()};
      w.full_planes = true;   // the captured run transforms every plane: warm the same cuFFT plans
      const int rc = rq->p->precision == 64 ? run_typed<double, double2>(e, w, e->stream)
                                            : run_typed<float, float2>(e, w, e->stream);
      if (rc) {
        m.status = fail(c, rc, std::string("batch: ") + e->err);
        m.ok = false;
      } else {
        e->graph_warm.insert(key);
      }
    }
  }
  // pinned host areas
  size_t total = 0;
  auto sizes = [&](const Request &rq, Pending &pd) {
    const int NL = rq.p->ell_max / 2 + 1;
    pd.host_len =
        sizeof(double) * (8 + (size_t)NL * (rq.kb ? rq.kb->nbins : 1) + (size_t)NL * (rq.rb ? rq.rb->nbins : 1));
    pd.stage_len = sizeof(double) * (size_t)(n_fields(rq.p) + 3 * rq.p->n_mesh + 2);   // scale, 1/W, phases
    total += pd.host_len + pd.stage_len;
  };
  for (auto &m : B->it)
    if (m.ok) {
      sizes(m.rq, m.pd);
      if (!m.rr.empty()) sizes(m.rrq, m.pdr);
    }
  if (total && cudaMallocHost((void **)&B->pinned, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "batch: pinned host allocation failed");
  }
  size_t off = 0;
  auto place = [&](Pending &pd) {
    pd.host = (double *)(B->pinned + off);
    off += pd.host_len;
    pd.stage = B->pinned + off;
    off += pd.stage_len;
  };
  for (auto &m : B->it)
    if (m.ok) {
      place(m.pd);
      if (!m.rr.empty()) place(m.pdr);
    }
  // capture (forked into one branch per engine, joined at the end) and instantiate
  bool setup = cudaStreamSynchronize(st) == cudaSuccess &&
               cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking) == cudaSuccess;
  for (int b = 0; setup && b < nb; ++b) {
    cudaStream_t q = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    setup = cudaStreamSynchronize(B->eng[(size_t)b]->stream) == cudaSuccess &&
            cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess;
    if (q) B->bst.push_back(q);
    if (e0) B->ev.push_back(e0);
    if (e1) B->ev.push_back(e1);
  }
  if (!setup) return fail(c, BYM_E_CUDA, "batch: capture streams");
  int rc = BYM_OK;
  if (cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    rc = fail(c, BYM_E_CUDA, "batch: stream capture could not start");
  } else {
    for (int b = 0; b < nb && !rc; ++b)   // fork
      if (cudaEventRecord(B->ev[2 * b], B->cs) != cudaSuccess || cudaStreamWaitEvent(B->bst[b], B->ev[2 * b], 0))
        rc = fail(c, BYM_E_CUDA, "batch: fork");
    for (auto &m : B->it) {
      if (!m.ok || rc) continue;
      bym_ctx *e = B->eng[(size_t)m.branch];
      cudaStream_t q = B->bst[(size_t)m.branch];
      const bool prof_was = e->prof;
      e->prof = false;
      const auto enq = [&](const Request &rq, Pending *pd) {
        return rq.p->precision == 64 ? run_typed<double, double2>(e, rq, q, pd)
                                     : run_typed<float, float2>(e, rq, q, pd);
      };
      rc = enq(m.rq, &m.pd);
      if (!rc && !m.rr.empty()) rc = enq(m.rrq, &m.pdr);
      e->prof = prof_was;
      if (rc) rc = fail(c, rc, std::string("batch: ") + e->err);
    }
    for (int b = 0; b < nb && !rc; ++b)   // join
      if (cudaEventRecord(B->ev[2 * b + 1], B->bst[b]) != cudaSuccess ||
          cudaStreamWaitEvent(B->cs, B->ev[2 * b + 1], 0) != cudaSuccess)
        rc = fail(c, BYM_E_CUDA, "batch: join");
    const cudaError_t ec = cudaStreamEndCapture(B->cs, &B->graph);
    if (!rc && ec != cudaSuccess) rc = fail(c, BYM_E_CUDA, std::string("batch: capture: ") + cudaGetErrorString(ec));
  }
  if (!rc && cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess)
    rc = fail(c, BYM_E_CUDA, std::string("batch: graph instantiation: ") + cudaGetErrorString(cudaGetLastError()));
  if (rc) return rc;
  out = std::move(B);
  return BYM_OK;
}

static int batch_launch(bym_batch *B, int *status) {
  bym_ctx *c = B->c;
  int first_err = BYM_OK;
  int rc = BYM_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) rc = fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  // the graph's buffers come from the graph memory pool: hand back what the stream-ordered
  // pool holds unused (it keeps freed memory between requests) before the launch maps them
  cudaMemPool_t pool;
  if (!rc && cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    cudaStreamSynchronize(c->stream);
    cudaMemPoolTrimTo(pool, 0);
  }
  if (!rc && cudaGraphLaunch(B->exec, B->cs) != cudaSuccess)
    rc = fail(c, BYM_E_CUDA, std::string("batch: graph launch: ") + cudaGetErrorString(cudaGetLastError()));
  if (!rc && cudaStreamSynchronize(B->cs) != cudaSuccess)
    rc = fail(c, BYM_E_CUDA, std::string("batch: graph run: ") + cudaGetErrorString(cudaGetLastError()));
  for (size_t i = 0; i < B->it.size(); ++i) {
    auto &m = B->it[i];
    int r = m.status;
    if (m.ok && rc) r = rc;
    if (m.ok && !rc) {
      const Pending &pd = m.pd;
      r = finish_results(c, m.rq, pd.host, pd.host + 8, pd.host + 8 + pd.NL * pd.nbk, pd.kg, pd.rg, pd.NL, pd.nbk,
                         pd.nbr, pd.h);
      if (!r && !m.rr.empty()) {
        const Pending &q = m.pdr;
        r = finish_results(c, m.rrq, q.host, q.host + 8, q.host + 8 + q.NL * q.nbk, q.kg, q.rg, q.NL, q.nbk, q.nbr,
                           q.h);
        const int nbr = m.rq.rb->nbins, NL = m.p.ell_max / 2 + 1;
        for (int b = 0; !r && b < nbr; ++b) {
          const double den = m.alpha * m.alpha * m.rr[(size_t)b];
          for (int l = 0; l < NL; ++l) m.rq.xi[l * nbr + b] = den != 0.0 ? m.rq.xi[l * nbr + b] / den : 0.0;
        }
      }
    }
    if (status) status[i] = r;
    if (r && !first_err) first_err = r;
  }
  return first_err;
}

int bym_batch_plan_create(bym_ctx *c, int n, const bym_request *reqs, const bym_result *outs, int n_streams,
                          bym_batch **plan, int *status) {
  if (!c || !plan || n < 0 || (n > 0 && (!reqs || !outs || !status))) return BYM_E_INVAL;
  *plan = nullptr;
  std::lock_guard<std::mutex> lock(c->mu);
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  std::unique_ptr<bym_batch> B;
  const int rc = batch_create(c, n, reqs, outs, n_streams, B);
  if (rc) return rc;
  int first_err = BYM_OK;
  for (int i = 0; i < n; ++i) {
    status[i] = B->it[(size_t)i].status;
    if (status[i] && !first_err) first_err = status[i];
  }
  *plan = B.release();
  return first_err;
}

int bym_batch_plan_launch(bym_batch *plan, int *status) {
  if (!plan) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(plan->c->mu);
  return batch_launch(plan, status);
}

void bym_batch_plan_destroy(bym_batch *plan) {
  if (!plan) return;
  bym_ctx *c = plan->c;
  std::lock_guard<std::mutex> lock(c->mu);
  delete plan;
}

int bym_batch_graph(bym_ctx *c, int n, const bym_request *reqs, const bym_result *outs, int *status) {
  if (!c || n < 0 || (n > 0 && (!reqs || !outs || !status))) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  std::unique_ptr<bym_batch> B;
  const int rc = batch_create(c, n, reqs, outs, 0, B);
  if (rc) {
    for (int i = 0; i < n; ++i) status[i] = rc;
    return rc;
  }
  return batch_launch(B.get(), status);
}

int bym_shot_noise(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                   double *shot) {
  if (!c || !shot) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  int rc = validate(c, gal, ran, p, nullptr, nullptr);
  if (rc) return rc;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  cudaStream_t st = c->stream;
  DevBufs buf(st);
  const bym_catalog *cats[2] = {gal, ran};
  double *stats = nullptr;
  if (buf.alloc((void **)&stats, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "device allocation failed");
  }
  cudaMemsetAsync(stats, 0, 8 * sizeof(double), st);
  const double inv_h = p->n_mesh / p->box_len;
  double *npart = nullptr;
  if (buf.alloc((void **)&npart, norm_scratch_bytes(c->nsm)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BYM_E_NOMEM, "device allocation failed");
  }
  for (int w = 0; w < 2; ++w) {
    const bym_catalog *cat = cats[w];
    if (!cat || cat->n <= 0) continue;
    const float4 *d4 = (const float4 *)cat->xyzw;
    const float *dn = cat->nbar;
    if (!cat->on_device) {
      void *a = nullptr, *b = nullptr;
      if (buf.alloc(&a, (size_t)cat->n * 16) != cudaSuccess ||
          (cat->nbar && buf.alloc(&b, (size_t)cat->n * 4) != cudaSuccess)) {
        cudaGetLastError();
        return fail(c, BYM_E_NOMEM, "device allocation failed");
      }
      cudaMemcpyAsync(a, cat->xyzw, (size_t)cat->n * 16, cudaMemcpyHostToDevice, st);
      if (cat->nbar) cudaMemcpyAsync(b, cat->nbar, (size_t)cat->n * 4, cudaMemcpyHostToDevice, st);
      d4 = (const float4 *)a;
      dn = (const float *)b;
    }
    launch_norm_reduce(d4, dn, cat->n, w, p->box_lo, inv_h, p->n_mesh, stats, npart, c->nsm, st, p->precision);
  }
  double hs[8];
  cudaError_t e = cudaMemcpyAsync(hs, stats, sizeof hs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, BYM_E_CUDA, std::string("shot noise: ") + cudaGetErrorString(e));
  if (hs[3] > 0.0)
    return fail(c, BYM_E_OUT_OF_BOX, std::to_string((long long)hs[3]) + " objects lie outside the box or are not finite");
  const double alpha = hs[1] != 0.0 ? hs[0] / hs[1] : 0.0;
  double S = hs[4] + alpha * alpha * hs[5];
  if (p->norm >= 1) {
    const double A = alpha * hs[2];
    if (!(A > 0.0) || !std::isfinite(A)) return fail(c, BYM_E_INVAL, "FKP normalisation A is not positive");
    S /= A;
  }
  *shot = S;
  return BYM_OK;
}

int bym_set_field_chunk(bym_ctx *c, int max_fields) {
  if (!c || max_fields < 0) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  c->field_chunk = max_fields;
  c->graph_warm.clear();
  return BYM_OK;
}

int bym_fft3d(bym_ctx *c, void *data, int n_mesh, int count, int inverse, void *stream) {
  if (!c || !data || count < 0 || n_mesh < 8 || n_mesh % 2) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  const size_t slot_bytes = (size_t)n_mesh * n_mesh * (n_mesh + kRowPad) * sizeof(float);
  int rc = fft_slots(c, st, 32, inverse ? 1 : 0, n_mesh, data, slot_bytes, 0, count, Tune());
  if (rc) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(c, BYM_E_CUDA, "FFT failed");
  prof_collect(c);
  return BYM_OK;
}

// Autotuner: time real runs of the caller's request under candidate launch
// shapes (per-kernel times from the tracer) and keep the fastest per kernel.
int bym_autotune(bym_ctx *c, const bym_catalog *gal, const bym_catalog *ran, const bym_params *p,
                 const bym_bins *kbins, const bym_bins *rbins, const char *cache_path, char *report,
                 size_t report_len) {
  if (!c || !p) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  int rc = validate(c, gal, ran, p, kbins, rbins);
  if (rc) return rc;
  const auto key = std::make_tuple(p->n_mesh, p->precision, p->los);
  char keybuf[96];
  snprintf(keybuf, sizeof keybuf, "n%d_p%d_los%d", p->n_mesh, p->precision, p->los);
  auto emit = [&](const Tune &t, const char *source) {
    if (!report || !report_len) return;
    char buf[512];
    snprintf(buf, sizeof buf,
             "{\"key\": \"%s\", \"source\": \"%s\", \"per_sm_gen\": %d, \"per_sm_comb\": %d, "
             "\"per_sm_k\": %d, \"per_sm_spec\": %d, \"fft_batch\": %d, \"native_fft\": %d}",
             keybuf, source, t.per_sm_gen, t.per_sm_comb, t.per_sm_k, t.per_sm_spec, t.fft_batch, t.native);
    snprintf(report, report_len, "%s", buf);
  };
  if (cache_path) {   // "key per_sm_gen per_sm_comb per_sm_k per_sm_spec fft_batch native" lines
    if (FILE *f = fopen(cache_path, "r")) {
      char k[96];
      Tune t;
      while (fscanf(f, "%95s %d %d %d %d %d %d", k, &t.per_sm_gen, &t.per_sm_comb, &t.per_sm_k, &t.per_sm_spec,
                    &t.fft_batch, &t.native) == 7) {
        if (strcmp(k, keybuf) == 0) {
          fclose(f);
          c->tune[key] = t;
          c->graph_warm.clear();
          emit(t, "cache");
          return BYM_OK;
        }
      }
      fclose(f);
    }
  }
  const bool want_pk = kbins != nullptr, want_xi = rbins != nullptr;
  const int NL = p->ell_max / 2 + 1;
  std::vector<double> pk(want_pk ? NL * kbins->nbins : 0), km(want_pk ? kbins->nbins : 0),
      xi(want_xi ? NL * rbins->nbins : 0), rm(want_xi ? rbins->nbins : 0);
  std::vector<int64_t> nm(want_pk ? kbins->nbins : 0), nc(want_xi ? rbins->nbins : 0);
  Request rq{gal, ran, p, kbins, rbins, want_pk ? pk.data() : nullptr, want_pk ? km.data() : nullptr,
             want_pk ? nm.data() : nullptr, want_xi ? xi.data() : nullptr, want_xi ? rm.data() : nullptr,
             want_xi ? nc.data() : nullptr};
  const bool prof_was = c->prof;
  auto timed = [&](const Tune &t, std::map<std::string, ProfEntry> &out) -> int {
    c->tune[key] = t;
    c->prof_tab.clear();
    c->prof = true;
    int r = run_request(c, rq, c->stream);
    c->prof = prof_was;
    out = c->prof_tab;
    c->prof_tab.clear();
    return r;
  };
  std::map<std::string, ProfEntry> prof;
  Tune best;
  if ((rc = timed(best, prof))) return rc;   // warm: kernels, plans, tables
  // grid shapes: one run per blocks-per-SM factor, best factor per kernel
  const int factors[] = {2, 4, 8, 16, 32};
  double bgen = 1e300, bcomb = 1e300, bk = 1e300, bspec = 1e300;
  for (int f : factors) {
    Tune t = best;
    t.per_sm_gen = t.per_sm_comb = t.per_sm_k = t.per_sm_spec = f;
    if ((rc = timed(t, prof))) return rc;
    for (auto &kv : prof) {
      const std::string &n = kv.first;
      const double ms = kv.second.ms;
      if (n.rfind("gen_fields", 0) == 0 && ms < bgen) bgen = ms, best.per_sm_gen = f;
      if (n == "mid_combine" && ms < bcomb) bcomb = ms, best.per_sm_comb = f;
      if (n.rfind("kcontract", 0) == 0 && ms < bk) bk = ms, best.per_sm_k = f;
      if (n == "spec_mul" && ms < bspec) bspec = ms, best.per_sm_spec = f;
    }
  }
  // transforms: library kernels against cuFFT, then cuFFT's batch size.  Every kernel whose work
  // depends on the choice is counted: the transforms, the spectral product, the occupied-plane scan
  // and the field generation (which writes only the occupied planes when the x pass reads only those)
  auto fft_ms = [](const std::map<std::string, ProfEntry> &m) {
    double s = 0.0;
    for (auto &kv : m)
      if (kv.first.rfind("cufft", 0) == 0 || kv.first.rfind("fft_native", 0) == 0 || kv.first == "spec_mul" ||
          kv.first == "plane_range" || kv.first.rfind("gen_fields", 0) == 0)
        s += kv.second.ms;
    return s;
  };
  double best_fft = 1e300;
  for (int b : {4, 8, 16}) {
    Tune t = best;
    t.native = 0;
    t.fft_batch = b;
    if ((rc = timed(t, prof))) return rc;
    const double ms = fft_ms(prof);
    if (ms < best_fft) best_fft = ms, best.fft_batch = b, best.native = 0;
  }
  if (c->fft_mode == 2) {   // cuFFT planes (forward over the occupied planes) + cuFFT along x
    Tune t = best;
    t.native = 2;
    if ((rc = timed(t, prof))) return rc;
    const double ms = fft_ms(prof);
    if (ms < best_fft) best_fft = ms, best.native = 2;
  }
  if (native_fft_supported(p->n_mesh, p->precision) && c->fft_mode == 2) {
    // cuFFT planes + library x pass; library z, y and x passes; library two-pass with 8- / 16-CTA clusters
    for (int cl : {1, 3, 8, 16}) {
      Tune t = best;
      t.native = cl;
      if ((rc = timed(t, prof))) return rc;
      const double ms = fft_ms(prof);
      if (ms < best_fft) best_fft = ms, best.native = cl;
    }
  }
  c->tune[key] = best;
  c->graph_warm.clear();
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "a")) {
      fprintf(f, "%s %d %d %d %d %d %d\n", keybuf, best.per_sm_gen, best.per_sm_comb, best.per_sm_k,
              best.per_sm_spec, best.fft_batch, best.native);
      fclose(f);
    }
  }
  emit(best, "measured");
  return BYM_OK;
}

int bym_profile_enable(bym_ctx *c, int enable) {
  if (!c) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  c->prof = enable != 0;
  return BYM_OK;
}

int bym_profile_read(bym_ctx *c, char *json, size_t len, int reset) {
  if (!c || !json || !len) return BYM_E_INVAL;
  std::lock_guard<std::mutex> lock(c->mu);
  std::ostringstream o;
  o.precision(17);
  o << "{";
  bool first = true;
  for (auto &kv : c->prof_tab) {
    o << (first ? "" : ", ") << "\"" << kv.first << "\": {\"launches\": " << kv.second.launches
      << ", \"ms\": " << kv.second.ms << ", \"bytes\": " << kv.second.bytes << "}";
    first = false;
  }
  o << "}";
  const std::string s = o.str();
  const size_t n = std::min(len - 1, s.size());
  memcpy(json, s.data(), n);
  json[n] = '\0';
  if (reset) c->prof_tab.clear();
  return s.size() < len ? BYM_OK : BYM_E_INVAL;
}

int bym_jit_check(const bym_params *p, char *log, size_t log_len) {
  if (!p) return BYM_E_INVAL;
  int rc = validate_params(nullptr, p);
  if (rc) return rc;
  std::string src, lg;
  try {
    src = generate_source(JitKey{p->los, p->ell_max, order_key(p), p->precision}, nullptr);
  } catch (const std::exception &e) {
    lg = e.what();
  }
  std::vector<char> cubin;
  bool ok = !src.empty() && compile_cubin(src, cubin, lg);
  if (ok && (is_midpoint(p) || p->los == BYM_LOS_BISECTOR)) {   // the field-range kernels too (16 fields)
    src.clear();
    try {
      src = generate_chunk_source(JitKey{p->los, p->ell_max, order_key(p), p->precision}, 16, nullptr);
    } catch (const std::exception &e) {
      lg = e.what();
    }
    ok = !src.empty() && compile_cubin(src, cubin, lg);
  }
  if (ok && p->los != BYM_LOS_MIDPOINT_EVEN && p->ell_max + 1 <= 7) {
    src.clear();   // the odd-multipole module for ell_max + 1
    try {
      src = generate_odd_source(JitKey{p->los, p->ell_max + 1, order_key(p), p->precision}, nullptr);
    } catch (const std::exception &e) {
      lg = e.what();
    }
    ok = !src.empty() && compile_cubin(src, cubin, lg);
  }
  if (ok && p->los == BYM_LOS_BISECTOR) {   // and the two-tracer contraction
    src.clear();
    try {
      src = generate_cross_source(JitKey{p->los, p->ell_max, order_key(p), p->precision});
    } catch (const std::exception &e) {
      lg = e.what();
    }
    ok = !src.empty() && compile_cubin(src, cubin, lg);
  }
  if (log && log_len) {
    const size_t n = std::min(log_len - 1, lg.size());
    memcpy(log, lg.data(), n);
    log[n] = '\0';
  }
  return ok ? BYM_OK : BYM_E_CUDA;
}

}  // extern "C"
