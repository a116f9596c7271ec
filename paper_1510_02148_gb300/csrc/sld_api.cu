// sld_api.cu -- the C ABI of libsld (declared in include/sld.h): handle
// lifetime, argument checks, host/device pointer marshalling, and the calls
// into the setup and solve launchers.  No arithmetic of the method runs here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sld_internal.h"

struct sld_batch_s {
  std::vector<sld_system> sys;
  sld_options o{};
  sld::BatchPlan plan;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t stream = nullptr;  // owned: graph capture and launch
  std::string desc;
};

namespace {

thread_local std::string g_last_error;

sld_status fail(sld_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

sld_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SLD_ERR_OOM : SLD_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_in(const void* src) {
  return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(const void* dst) {
  return is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

// Relative Cholesky pivot bound for the extra dense columns: a pivot below
// this fraction of its diagonal means the column is numerically in the span
// of the others (E would be near-singular), and the extra columns are dropped.
constexpr double kLearnedPivotTol = 1e-10;

__global__ void k_count_bad_K(int64_t n, const double* __restrict__ K, unsigned long long* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double k = K[i];
    if (!(k > 0.0) || !isfinite(k)) atomicAdd(bad, 1ull);
  }
}

sld_status ensure_workspace(sld_system s, bool need_fp32, bool need_bf16) {
  const int64_t n = s->g.n;
  cudaError_t e;
  if (!s->x) {
    if ((e = dalloc(&s->x, n)) != cudaSuccess) return cuda_fail(e, "alloc x");
    if ((e = dalloc(&s->r64, n)) != cudaSuccess) return cuda_fail(e, "alloc r");
    if ((e = dalloc(&s->bwork, n)) != cudaSuccess) return cuda_fail(e, "alloc b");
    // inner vectors: n FP64 (FP64 form, rows unpadded) or np FP32 (padded rows)
    const int64_t nv = std::max<int64_t>(n, (s->np + 1) / 2);
    s->nvec = nv;
    double* v[4];
    for (int k = 0; k < 4; ++k)
      if ((e = dalloc(&v[k], nv)) != cudaSuccess) return cuda_fail(e, "alloc vectors");
    s->z = v[0];
    s->p0 = v[1];
    s->p1 = v[2];
    s->xh = v[3];
    if ((e = dalloc(&s->out, 64)) != cudaSuccess) return cuda_fail(e, "alloc out");
    if ((e = dalloc(&s->bar, 64)) != cudaSuccess) return cuda_fail(e, "alloc barrier");
    if ((e = dalloc(&s->status, 16)) != cudaSuccess) return cuda_fail(e, "alloc status");
  }
  if (s->part_rows == 0 || !s->part) {
    s->part_rows = s->nsm * 8;
    const int pstride = (sld::kMaxD + sld::kMaxL + sld::kPartScalars + 3) / 4 * 4;
    if ((e = dalloc(&s->part, (size_t)s->part_rows * pstride)) != cudaSuccess) return cuda_fail(e, "alloc partials");
    if ((e = dalloc(&s->s_glob, sld::kMaxD + sld::kMaxL + sld::kPartScalars)) != cudaSuccess)
      return cuda_fail(e, "alloc s");
    if ((e = dalloc(&s->y_glob, sld::kMaxD + sld::kMaxL + sld::kPartScalars)) != cudaSuccess)
      return cuda_fail(e, "alloc y");
  }
  if (need_fp32 && !s->Tx32) {
    // all three or none, so that a failed allocation leaves no half-made set
    float *tx = nullptr, *ty = nullptr, *tz = nullptr;
    if ((e = dalloc(&tx, s->np)) != cudaSuccess || (e = dalloc(&ty, s->np)) != cudaSuccess ||
        (e = dalloc(&tz, s->np)) != cudaSuccess) {
      dfree(tx);
      dfree(ty);
      dfree(tz);
      cudaGetLastError();
      return cuda_fail(e, "alloc FP32 faces");
    }
    s->Tx32 = tx;
    s->Ty32 = ty;
    s->Tz32 = tz;
    if ((e = sld::launch_quantize_fp32(s)) != cudaSuccess) return cuda_fail(e, "fp32 coefficients");
  }
  if (need_bf16 && !s->bf16_ready) {
    // BF16 faces, their FP32 inverse diagonal, and E = Z^T A16 Z of the
    // quantized operator with its inverse (the inner iterations deflate with
    // the operator they apply)
    if (!s->Tx16) {
      if ((e = dalloc(&s->Tx16, s->np)) != cudaSuccess) return cuda_fail(e, "alloc Tx16");
      if ((e = dalloc(&s->Ty16, s->np)) != cudaSuccess) return cuda_fail(e, "alloc Ty16");
      if ((e = dalloc(&s->Tz16, s->np)) != cudaSuccess) return cuda_fail(e, "alloc Tz16");
      if ((e = dalloc(&s->invd16, s->np)) != cudaSuccess) return cuda_fail(e, "alloc invd16");
    }
    dfree(s->E16);
    dfree(s->Einv16);
    s->E16 = s->Einv16 = nullptr;
    if ((e = dalloc(&s->E16, (size_t)s->d * s->d)) != cudaSuccess) return cuda_fail(e, "alloc E16");
    if ((e = dalloc(&s->Einv16, (size_t)s->d * s->d)) != cudaSuccess) return cuda_fail(e, "alloc Einv16");
    if ((e = sld::launch_quantize_bf16(s)) != cudaSuccess) return cuda_fail(e, "bf16 coefficients");
    double* wide = nullptr;
    if ((e = dalloc(&wide, 3 * (size_t)n)) != cudaSuccess) return cuda_fail(e, "alloc widened faces");
    int bad = 0;
    e = sld::launch_widen_bf16(s, wide, wide + n, wide + 2 * n);
    if (e == cudaSuccess) e = sld::launch_coarse_E(s, wide, wide + n, wide + 2 * n, s->E16, &bad);
    dfree(wide);
    if (e != cudaSuccess) return cuda_fail(e, "bf16 coarse matrix");
    std::string msg;
    const int st = sld::coarse_factor(s, s->d, s->E16, s->Einv16, 2.0, &msg);
    if (st != SLD_OK) return fail((sld_status)st, "bf16 coarse matrix: " + msg);
    s->bf16_ready = true;
  }
  return SLD_OK;
}

}  // namespace

namespace sld {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace sld

extern "C" {

void sld_default_options(sld_options* o) {
  if (!o) return;
  o->precision = SLD_FP64;
  o->tol = 1e-9;
  o->inner_tol = 1e-5;
  o->maxiter = 20000;
  o->max_outer = 40;
  o->ctas_per_sm = 0;
  o->timeout_s = 2.0;
  o->debug_skip_barrier = -1;
  o->fwd_tol = 0.0;
}

const char* sld_last_error(void) { return g_last_error.c_str(); }

sld_status sld_build_system(const double* K, const double* q, sld_grid g, sld_bc bc, void* stream,
                            sld_system* out) {
  g_last_error.clear();
  if (!out) return fail(SLD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!K) return fail(SLD_ERR_INVALID_ARG, "K is NULL");
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(SLD_ERR_INVALID_ARG, "grid sizes must be >= 1");
  const int64_t n = (int64_t)g.nx * g.ny * g.nz;
  if (n > ((int64_t)1 << 31) - 1) return fail(SLD_ERR_INVALID_ARG, "more than 2^31-1 cells");
  bool anyd = false;
  for (int f = 0; f < 6; ++f) {
    if (bc.type[f] != SLD_BC_NOFLOW && bc.type[f] != SLD_BC_DIRICHLET)
      return fail(SLD_ERR_INVALID_ARG, "bc.type must be SLD_BC_NOFLOW or SLD_BC_DIRICHLET");
    if (bc.type[f] == SLD_BC_DIRICHLET) {
      anyd = true;
      if (!std::isfinite(bc.value[f])) return fail(SLD_ERR_INVALID_ARG, "Dirichlet value not finite");
    }
  }
  if (!anyd) return fail(SLD_ERR_INVALID_ARG, "at least one Dirichlet face is needed (A singular otherwise)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return cuda_fail(e, "device properties");
  if (prop.major != 10 || prop.minor != 3)
    return fail(SLD_ERR_CUDA, "libsld is built for sm_103 (GB300) only; device is sm_" +
                                  std::to_string(prop.major) + std::to_string(prop.minor));
  if (!prop.cooperativeLaunch) return fail(SLD_ERR_CUDA, "device without cooperative launch");
  sld_system s = new sld_system_s();
  s->device = dev;
  s->nsm = prop.multiProcessorCount;
  s->stream = static_cast<cudaStream_t>(stream);
  s->g.nx = g.nx;
  s->g.ny = g.ny;
  s->g.nz = g.nz;
  s->g.nxy = (int64_t)g.nx * g.ny;
  s->g.n = n;
  s->nxp = (g.nx + 7) / 8 * 8;
  s->np = (int64_t)s->nxp * g.ny * g.nz;
  for (int f = 0; f < 6; ++f) {
    s->bc_type[f] = bc.type[f];
    s->bc_value[f] = bc.value[f];
  }
  s->g.dlo_x = bc.type[0] == SLD_BC_DIRICHLET;
  s->g.dhi_x = bc.type[1] == SLD_BC_DIRICHLET;
  s->g.dlo_y = bc.type[2] == SLD_BC_DIRICHLET;
  s->g.dhi_y = bc.type[3] == SLD_BC_DIRICHLET;
  s->g.dlo_z = bc.type[4] == SLD_BC_DIRICHLET;
  s->g.dhi_z = bc.type[5] == SLD_BC_DIRICHLET;
  double* qd = nullptr;
  unsigned long long* bad = nullptr;
  unsigned long long hbad = 0;
  sld_status st = SLD_OK;
  do {
    if ((e = dalloc(&s->K, n)) != cudaSuccess) { st = cuda_fail(e, "alloc K"); break; }
    if ((e = dalloc(&s->Tx, n)) != cudaSuccess) { st = cuda_fail(e, "alloc Tx"); break; }
    if ((e = dalloc(&s->Ty, n)) != cudaSuccess) { st = cuda_fail(e, "alloc Ty"); break; }
    if ((e = dalloc(&s->Tz, n)) != cudaSuccess) { st = cuda_fail(e, "alloc Tz"); break; }
    if ((e = dalloc(&s->diag, n)) != cudaSuccess) { st = cuda_fail(e, "alloc diag"); break; }
    if ((e = dalloc(&s->invdiag, n)) != cudaSuccess) { st = cuda_fail(e, "alloc invdiag"); break; }
    if ((e = dalloc(&s->b, n)) != cudaSuccess) { st = cuda_fail(e, "alloc b"); break; }
    if ((e = cudaEventCreate(&s->ev0)) != cudaSuccess) { st = cuda_fail(e, "event"); break; }
    if ((e = cudaEventCreate(&s->ev1)) != cudaSuccess) { st = cuda_fail(e, "event"); break; }
    if ((e = cudaMemcpyAsync(s->K, K, sizeof(double) * n, kind_in(K), s->stream)) != cudaSuccess) {
      st = cuda_fail(e, "copy K");
      break;
    }
    if (q) {
      if ((e = dalloc(&qd, n)) != cudaSuccess) { st = cuda_fail(e, "alloc q"); break; }
      if ((e = cudaMemcpyAsync(qd, q, sizeof(double) * n, kind_in(q), s->stream)) != cudaSuccess) {
        st = cuda_fail(e, "copy q");
        break;
      }
    }
    if ((e = dalloc(&bad, 1)) != cudaSuccess) { st = cuda_fail(e, "alloc"); break; }
    cudaMemsetAsync(bad, 0, sizeof(*bad), s->stream);
    k_count_bad_K<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(n, s->K, bad);
    cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s->stream);
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) { st = cuda_fail(e, "check K"); break; }
    if (hbad) {
      st = fail(SLD_ERR_INVALID_ARG, std::to_string(hbad) + " permeability values are <= 0 or not finite");
      break;
    }
    if ((e = sld::launch_assemble(s, qd)) != cudaSuccess) { st = cuda_fail(e, "assemble"); break; }
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) { st = cuda_fail(e, "assemble"); break; }
  } while (false);
  dfree(qd);
  dfree(bad);
  if (st != SLD_OK) {
    sld_destroy(s);
    return st;
  }
  *out = s;
  return SLD_OK;
}

namespace {
// the plain subdomain-levelset labels into s->label (argument checks included)
sld_status plain_labels(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L, int64_t dmax) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (Sx < 1 || Sy < 1 || Sz < 1 || Sx > s->g.nx || Sy > s->g.ny || Sz > s->g.nz)
    return fail(SLD_ERR_INVALID_ARG, "subdomain counts must be in [1, grid size]");
  if (L < 1 || L > 16) return fail(SLD_ERR_INVALID_ARG, "L must be in [1, 16]");
  if (L > 1 && !tau) return fail(SLD_ERR_INVALID_ARG, "tau is NULL");
  const int64_t d = (int64_t)Sx * Sy * Sz * L;
  if (d > dmax) return fail(SLD_ERR_INVALID_ARG, "d = Sx*Sy*Sz*L exceeds " + std::to_string(dmax));
  double htau[16] = {0};
  if (L > 1) {
    cudaError_t e = cudaMemcpy(htau, tau, sizeof(double) * (L - 1), is_device_ptr(tau) ? cudaMemcpyDeviceToHost
                                                                                         : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy tau");
    for (int m = 0; m < L - 1; ++m) {
      if (!std::isfinite(htau[m])) return fail(SLD_ERR_INVALID_ARG, "tau not finite");
      if (m > 0 && !(htau[m] > htau[m - 1])) return fail(SLD_ERR_INVALID_ARG, "tau must ascend strictly");
    }
  }
  cudaError_t e;
  if (!s->label && (e = dalloc(&s->label, s->g.n)) != cudaSuccess) return cuda_fail(e, "alloc labels");
  if ((e = sld::launch_labels(s, Sx, Sy, Sz, htau, L)) != cudaSuccess) return cuda_fail(e, "labels");
  s->have_labels_d = (int)d;
  s->labels_L = L;
  s->deflation_ready = false;
  return SLD_OK;
}

sld_status labels_out_copy(sld_system s, int32_t* labels_out) {
  cudaError_t e;
  if (labels_out) {
    if ((e = cudaMemcpyAsync(labels_out, s->label, sizeof(int32_t) * s->g.n, kind_out(labels_out), s->stream)) !=
        cudaSuccess)
      return cuda_fail(e, "copy labels out");
  }
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "labels");
  return SLD_OK;
}

}  // namespace

sld_status sld_make_labels(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L, int32_t* labels_out) {
  g_last_error.clear();
  sld_status st = plain_labels(s, Sx, Sy, Sz, tau, L, sld::kMaxD);
  if (st != SLD_OK) return st;
  return labels_out_copy(s, labels_out);
}

sld_status sld_make_labels_cc(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L, int32_t* labels_out,
                              int* d_out) {
  g_last_error.clear();
  if (!d_out) return fail(SLD_ERR_INVALID_ARG, "d_out is NULL");
  sld_status st = plain_labels(s, Sx, Sy, Sz, tau, L, 1 << 20);
  if (st != SLD_OK) return st;
  std::string msg;
  int d = 0;
  const int code = sld::run_cc_labels(s, s->have_labels_d, sld::kMaxD, &d, &msg);
  *d_out = d;
  if (code != SLD_OK) return fail((sld_status)code, msg);
  s->have_labels_d = d;
  s->labels_L = 0;  // component labels have no subdomain * L + class structure
  return labels_out_copy(s, labels_out);
}

sld_status sld_build_deflation(sld_system s, const int32_t* labels, int d, const void* Zextra, int k,
                               int zextra_dtype) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (k < 0 || k > sld::kMaxL) return fail(SLD_ERR_INVALID_ARG, "k must be in [0, " + std::to_string(sld::kMaxL) + "]");
  if ((k > 0) != (Zextra != nullptr)) return fail(SLD_ERR_INVALID_ARG, "Zextra must be given exactly when k > 0");
  if (k > 0 && zextra_dtype != SLD_ZEXTRA_F64 && zextra_dtype != SLD_ZEXTRA_F32)
    return fail(SLD_ERR_INVALID_ARG, "zextra_dtype must be SLD_ZEXTRA_F64 or SLD_ZEXTRA_F32");
  if (d < 1 || d > sld::kMaxD) return fail(SLD_ERR_INVALID_ARG, "d must be in [1, " + std::to_string(sld::kMaxD) + "]");
  cudaError_t e;
  if (labels) {
    if (!s->label && (e = dalloc(&s->label, s->g.n)) != cudaSuccess) return cuda_fail(e, "alloc labels");
    if ((e = cudaMemcpyAsync(s->label, labels, sizeof(int32_t) * s->g.n, kind_in(labels), s->stream)) != cudaSuccess)
      return cuda_fail(e, "copy labels");
    s->labels_L = 0;  // any labels: no subdomain structure assumed
  } else if (!s->label || s->have_labels_d == 0) {
    return fail(SLD_ERR_STATE, "no labels: pass them or call sld_make_labels first");
  }
  const int D = d + k;
  dfree(s->E);
  dfree(s->Einv);
  s->E = s->Einv = nullptr;
  if ((e = dalloc(&s->E, (size_t)D * D)) != cudaSuccess) return cuda_fail(e, "alloc E");
  if ((e = dalloc(&s->Einv, (size_t)D * D)) != cudaSuccess) return cuda_fail(e, "alloc Einv");
  s->d = d;
  s->kL = 0;
  s->kL_requested = k;
  s->deflation_ready = false;
  s->bf16_ready = false;
  int bad = 0;
  if ((e = sld::launch_coarse_E(s, s->Tx, s->Ty, s->Tz, s->E, &bad)) != cudaSuccess)
    return cuda_fail(e, "coarse matrix");
  if (bad) return fail(SLD_ERR_INVALID_ARG, "a label is outside [0, d)");
  if (!s->label16 && (e = dalloc(&s->label16, s->np)) != cudaSuccess) return cuda_fail(e, "alloc labels16");
  if ((e = sld::launch_labels16(s)) != cudaSuccess) return cuda_fail(e, "labels16");
  std::string msg;
  if (k > 0) {
    // Z = [Z_lab, Z_L]: E with the extra blocks, factored with a relative
    // pivot bound on the extra columns; if that fails the extra columns are
    // dropped and the plain label deflation is built instead.
    const int64_t n = s->g.n;
    if (!s->ZL32) {
      if ((e = dalloc(&s->ZL32, (size_t)n * sld::kMaxL)) != cudaSuccess) return cuda_fail(e, "alloc Z_L");
      if ((e = dalloc(&s->WL64, (size_t)n * sld::kMaxL)) != cudaSuccess) return cuda_fail(e, "alloc W_L");
      if ((e = dalloc(&s->WL32, (size_t)n * sld::kMaxL)) != cudaSuccess) return cuda_fail(e, "alloc W_L32");
    }
    const size_t zbytes = (zextra_dtype == SLD_ZEXTRA_F32 ? 4 : 8) * (size_t)n * k;
    const void* zsrc = Zextra;
    void* staged = nullptr;
    if (!is_device_ptr(Zextra)) {
      if ((e = cudaMalloc(&staged, zbytes)) != cudaSuccess) return cuda_fail(e, "alloc Zextra staging");
      if ((e = cudaMemcpyAsync(staged, Zextra, zbytes, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) {
        cudaFree(staged);
        return cuda_fail(e, "copy Zextra");
      }
      zsrc = staged;
    }
    double* Ef = nullptr;
    if ((e = dalloc(&Ef, (size_t)D * D)) != cudaSuccess) {
      if (staged) cudaFree(staged);
      return cuda_fail(e, "alloc E");
    }
    int zbad = 0;
    e = sld::launch_learned_setup(s, zsrc, k, zextra_dtype == SLD_ZEXTRA_F32, s->E, Ef, &zbad);
    if (staged) cudaFree(staged);
    if (e != cudaSuccess) {
      dfree(Ef);
      return cuda_fail(e, "extra vectors");
    }
    if (zbad) {
      dfree(Ef);
      return fail(SLD_ERR_INVALID_ARG, "Zextra holds a non-finite value");
    }
    s->kL = k;
    const int st = sld::coarse_factor(s, D, Ef, s->Einv, 2.0, &msg, d, kLearnedPivotTol);
    if (st == SLD_OK) {
      cudaMemcpyAsync(s->E, Ef, sizeof(double) * D * D, cudaMemcpyDeviceToDevice, s->stream);
      e = cudaStreamSynchronize(s->stream);
      dfree(Ef);
      if (e != cudaSuccess) return cuda_fail(e, "copy E");
      s->deflation_ready = true;
      return SLD_OK;
    }
    dfree(Ef);
    if (st != SLD_ERR_COARSE_SINGULAR) return fail((sld_status)st, msg);
    s->kL = 0;  // fall back to the label columns alone
    msg.clear();
  }
  const int st = sld::coarse_factor(s, d, s->E, s->Einv, 2.0, &msg);
  if (st != SLD_OK) return fail((sld_status)st, msg);
  s->deflation_ready = true;
  return SLD_OK;
}

sld_status sld_deflation_info(sld_system s, int* d, int* k_requested, int* k_used) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (!s->deflation_ready) return fail(SLD_ERR_STATE, "no deflation built");
  if (d) *d = s->d;
  if (k_requested) *k_requested = s->kL_requested;
  if (k_used) *k_used = s->kL;
  return SLD_OK;
}

sld_status sld_solve(sld_system s, const double* b, const sld_options* opt, double* x, sld_result* res) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (!x) return fail(SLD_ERR_INVALID_ARG, "x is NULL");
  if (!s->deflation_ready) return fail(SLD_ERR_STATE, "call sld_build_deflation before sld_solve");
  sld_options o;
  sld_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != SLD_FP64 && o.precision != SLD_FP32_IR && o.precision != SLD_BF16COEF_IR)
    return fail(SLD_ERR_INVALID_ARG, "precision must be SLD_FP64, SLD_FP32_IR or SLD_BF16COEF_IR");
  if (!(o.tol > 0) || !(o.tol < 1)) return fail(SLD_ERR_INVALID_ARG, "tol must be in (0, 1)");
  if (!(o.inner_tol > 0) || !(o.inner_tol < 1)) return fail(SLD_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
  if (!std::isfinite(o.fwd_tol)) return fail(SLD_ERR_INVALID_ARG, "fwd_tol must be finite");
  if (o.maxiter < 1 || o.max_outer < 1) return fail(SLD_ERR_INVALID_ARG, "maxiter and max_outer must be >= 1");
  sld_status st = ensure_workspace(s, o.precision == SLD_FP32_IR, o.precision == SLD_BF16COEF_IR);
  if (st != SLD_OK) return st;
  const int64_t n = s->g.n;
  const double* bd = s->b;
  cudaError_t e;
  if (b) {
    if (is_device_ptr(b)) {
      bd = b;
    } else {
      if ((e = cudaMemcpyAsync(s->bwork, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        return cuda_fail(e, "copy b");
      bd = s->bwork;
    }
  }
  cudaMemsetAsync(s->status, 0, sizeof(int) * 4, s->stream);
  sld_result r{};
  std::string msg;
  int code = sld::run_solve(s, bd, o, &r, &msg);
  if (code == SLD_ERR_CUDA || code == SLD_ERR_TIMEOUT || code < 0) {
    if (res) *res = r;
    return fail(code < 0 ? SLD_ERR_CUDA : (sld_status)code, msg);
  }
  // BF16 coefficients whose forward-error test gave up above fwd_tol (the
  // residual test met): the quantised operator does not resolve the slowest
  // modes of this field, so the solve goes on from its x with FP32-inner
  // refinement steps (the FP32 faces are made on first use).
  const double fwd_eff = o.fwd_tol == 0.0 ? 100.0 * o.tol : o.fwd_tol;
  bool hand_on = code == SLD_OK && o.precision == SLD_BF16COEF_IR && o.fwd_tol >= 0.0 && r.fwd_err_estimate > fwd_eff;
  if (hand_on && ensure_workspace(s, true, false) != SLD_OK) {
    // no room for the FP32 faces: the BF16 result stands (its estimate above
    // fwd_tol tells the caller)
    hand_on = false;
    g_last_error.clear();
    cudaGetLastError();
  }
  if (hand_on) {
    sld_options o2 = o;
    o2.precision = SLD_FP32_IR;
    sld_result r2{};
    cudaMemsetAsync(s->status, 0, sizeof(int) * 4, s->stream);
    code = sld::run_solve(s, bd, o2, &r2, &msg, true);
    r.iterations += r2.iterations;
    r.outer_steps += r2.outer_steps;
    r.solve_ms += r2.solve_ms;
    r.recursive_relres = r2.recursive_relres;
    r.fwd_err_estimate = r2.fwd_err_estimate;
    if (code == SLD_ERR_CUDA || code == SLD_ERR_TIMEOUT || code < 0) {
      if (res) *res = r;
      return fail(code < 0 ? SLD_ERR_CUDA : (sld_status)code, msg);
    }
  }
  double rr = 0, bb = 0;
  if ((e = sld::launch_residual(s, bd, s->x, s->part, &rr, &bb)) != cudaSuccess) return cuda_fail(e, "residual");
  r.true_relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if ((e = cudaMemcpyAsync(x, s->x, sizeof(double) * n, kind_out(x), s->stream)) != cudaSuccess)
    return cuda_fail(e, "copy x out");
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "copy x out");
  if (res) *res = r;
  if (code != SLD_OK) return fail((sld_status)code, msg);
  return SLD_OK;
}

sld_status sld_solve_gmres(sld_system s, const double* b, int m, int deflate, double tol, int maxiter, double* x,
                           sld_gmres_info* info) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (!x) return fail(SLD_ERR_INVALID_ARG, "x is NULL");
  if (m < 1 || m > 31) return fail(SLD_ERR_INVALID_ARG, "m must be in 1 .. 31");
  if (!(tol > 0) || !(tol < 1)) return fail(SLD_ERR_INVALID_ARG, "tol must be in (0, 1)");
  if (maxiter < 1) return fail(SLD_ERR_INVALID_ARG, "maxiter must be >= 1");
  if (deflate && !s->deflation_ready) return fail(SLD_ERR_STATE, "call sld_build_deflation before a deflated solve");
  if (deflate && s->kL > 0) return fail(SLD_ERR_STATE, "GMRES deflates with label columns only (no extra columns)");
  sld_status st = ensure_workspace(s, false, false);
  if (st != SLD_OK) return st;
  const int64_t n = s->g.n;
  const double* bd = s->b;
  cudaError_t e;
  if (b) {
    if (is_device_ptr(b)) {
      bd = b;
    } else {
      if ((e = cudaMemcpyAsync(s->bwork, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        return cuda_fail(e, "copy b");
      bd = s->bwork;
    }
  }
  sld_gmres_info r{};
  std::string msg;
  const int code = sld::run_gmres(s, bd, m, deflate ? 1 : 0, tol, maxiter, &r, &msg);
  if (code != SLD_OK && code != SLD_ERR_NOT_CONVERGED) {
    if (info) *info = r;
    return fail((sld_status)code, msg);
  }
  double rr = 0, bb = 0;
  if ((e = sld::launch_residual(s, bd, s->x, s->part, &rr, &bb)) != cudaSuccess) return cuda_fail(e, "residual");
  r.true_relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if ((e = cudaMemcpyAsync(x, s->x, sizeof(double) * n, kind_out(x), s->stream)) != cudaSuccess)
    return cuda_fail(e, "copy x out");
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "copy x out");
  if (info) *info = r;
  if (code != SLD_OK) return fail((sld_status)code, msg);
  return SLD_OK;
}

sld_status sld_solve_rdgmres(sld_system s, const double* b, int m, int d, double tol, int maxiter, double* x,
                             sld_gmres_info* info) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (!x) return fail(SLD_ERR_INVALID_ARG, "x is NULL");
  if (m < 2 || m > 31) return fail(SLD_ERR_INVALID_ARG, "m must be in 2 .. 31");
  if (d < 1 || d > 8 || d > m) return fail(SLD_ERR_INVALID_ARG, "d must be in 1 .. min(8, m)");
  if (!(tol > 0) || !(tol < 1)) return fail(SLD_ERR_INVALID_ARG, "tol must be in (0, 1)");
  if (maxiter < 1) return fail(SLD_ERR_INVALID_ARG, "maxiter must be >= 1");
  sld_status st = ensure_workspace(s, false, false);
  if (st != SLD_OK) return st;
  const int64_t n = s->g.n;
  const double* bd = s->b;
  cudaError_t e;
  if (b) {
    if (is_device_ptr(b)) {
      bd = b;
    } else {
      if ((e = cudaMemcpyAsync(s->bwork, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        return cuda_fail(e, "copy b");
      bd = s->bwork;
    }
  }
  sld_gmres_info r{};
  std::string msg;
  const int code = sld::run_rdgmres(s, bd, m, d, tol, maxiter, &r, &msg);
  if (code != SLD_OK && code != SLD_ERR_NOT_CONVERGED) {
    if (info) *info = r;
    return fail((sld_status)code, msg);
  }
  double rr = 0, bb = 0;
  if ((e = sld::launch_residual(s, bd, s->x, s->part, &rr, &bb)) != cudaSuccess) return cuda_fail(e, "residual");
  r.true_relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if ((e = cudaMemcpyAsync(x, s->x, sizeof(double) * n, kind_out(x), s->stream)) != cudaSuccess)
    return cuda_fail(e, "copy x out");
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "copy x out");
  if (info) *info = r;
  if (code != SLD_OK) return fail((sld_status)code, msg);
  return SLD_OK;
}

void sld_destroy(sld_system s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  void* ptrs[] = {s->K, s->Tx, s->Ty, s->Tz, s->diag, s->invdiag, s->b, s->Tx32, s->Ty32, s->Tz32,
                  s->Tx16, s->Ty16, s->Tz16, s->invd16, s->E16, s->Einv16,
                  s->label, s->label16, s->E, s->Einv, s->ZL32, s->WL64, s->WL32, s->x, s->r64, s->bwork, s->z, s->p0, s->p1, s->xh,
                  s->part, s->s_glob, s->y_glob, s->out, s->bar, s->status, s->gacc, s->gm_ws};
  for (void* p : ptrs) dfree(p);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  delete s;
}

sld_status sld_get_operator(sld_system s, double* Tx, double* Ty, double* Tz, double* diag, double* b) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  const size_t bytes = sizeof(double) * s->g.n;
  const double* src[5] = {s->Tx, s->Ty, s->Tz, s->diag, s->b};
  double* dst[5] = {Tx, Ty, Tz, diag, b};
  for (int k = 0; k < 5; ++k) {
    if (!dst[k]) continue;
    cudaError_t e = cudaMemcpyAsync(dst[k], src[k], bytes, kind_out(dst[k]), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy operator");
  }
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy operator");
  return SLD_OK;
}

sld_status sld_apply_A(sld_system s, const double* x, double* y) {
  g_last_error.clear();
  if (!s || !x || !y) return fail(SLD_ERR_INVALID_ARG, "NULL argument");
  const int64_t n = s->g.n;
  double *xd = nullptr, *yd = nullptr;
  cudaError_t e;
  if ((e = dalloc(&xd, n)) != cudaSuccess) return cuda_fail(e, "alloc");
  if ((e = dalloc(&yd, n)) != cudaSuccess) {
    dfree(xd);
    return cuda_fail(e, "alloc");
  }
  cudaMemcpyAsync(xd, x, sizeof(double) * n, kind_in(x), s->stream);
  e = sld::launch_apply_A(s, xd, yd);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, yd, sizeof(double) * n, kind_out(y), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(xd);
  dfree(yd);
  if (e != cudaSuccess) return cuda_fail(e, "apply A");
  return SLD_OK;
}

sld_status sld_restrict(sld_system s, const double* v, double* out) {
  g_last_error.clear();
  if (!s || !v || !out) return fail(SLD_ERR_INVALID_ARG, "NULL argument");
  if (!s->label || s->d < 1) return fail(SLD_ERR_STATE, "no deflation built");
  const int64_t n = s->g.n;
  double *vd = nullptr, *od = nullptr;
  cudaError_t e;
  if ((e = dalloc(&vd, n)) != cudaSuccess) return cuda_fail(e, "alloc");
  if ((e = dalloc(&od, s->d)) != cudaSuccess) {
    dfree(vd);
    return cuda_fail(e, "alloc");
  }
  cudaMemcpyAsync(vd, v, sizeof(double) * n, kind_in(v), s->stream);
  e = sld::launch_restrict(s, vd, od);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, od, sizeof(double) * s->d, kind_out(out), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(vd);
  dfree(od);
  if (e != cudaSuccess) return cuda_fail(e, "restrict");
  return SLD_OK;
}

sld_status sld_get_coarse(sld_system s, double* E, double* Einv) {
  g_last_error.clear();
  if (!s) return fail(SLD_ERR_INVALID_ARG, "handle is NULL");
  if (!s->E) return fail(SLD_ERR_STATE, "no deflation built");
  const size_t bytes = sizeof(double) * s->dk() * s->dk();
  cudaError_t e = cudaSuccess;
  if (E) e = cudaMemcpyAsync(E, s->E, bytes, kind_out(E), s->stream);
  if (e == cudaSuccess && Einv) e = cudaMemcpyAsync(Einv, s->Einv, bytes, kind_out(Einv), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy coarse");
  return SLD_OK;
}

}  // extern "C"

namespace {

// Results of system s after a solve that ended without a CUDA error.
sld_status collect(sld_system s, const double* b_dev, double ms, double* x, sld_result* r) {
  double out[sld::kOutCount];
  int dev_status = 0;
  cudaMemcpyAsync(out, s->out, sizeof(out), cudaMemcpyDeviceToHost, s->stream);
  cudaMemcpyAsync(&dev_status, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch readback");
  r->iterations = (int)out[sld::kOutIters];
  r->outer_steps = (int)out[sld::kOutOuter];
  r->recursive_relres = out[sld::kOutBB] > 0 ? std::sqrt(out[sld::kOutRecRR] / out[sld::kOutBB]) : 0.0;
  r->fwd_err_estimate = out[sld::kOutFwd];
  r->solve_ms = ms;
  r->kernel_path = 2;
  if (dev_status != 0) return fail((sld_status)dev_status, "a device-side wait timed out (team barrier)");
  double rr = 0, bb = 0;
  if ((e = sld::launch_residual(s, b_dev, s->x, s->part, &rr, &bb)) != cudaSuccess) return cuda_fail(e, "residual");
  r->true_relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if (x) {
    if ((e = cudaMemcpyAsync(x, s->x, sizeof(double) * s->g.n, kind_out(x), s->stream)) != cudaSuccess)
      return cuda_fail(e, "copy x out");
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "copy x out");
  }
  const int code = (int)out[sld::kOutStatus];
  if (code == SLD_ERR_NOT_CONVERGED) return fail(SLD_ERR_NOT_CONVERGED, "not converged within maxiter / max_outer");
  if (code == SLD_ERR_BREAKDOWN) return fail(SLD_ERR_BREAKDOWN, "breakdown in the deflated iteration");
  if (code < 0) return fail(SLD_ERR_CUDA, "device error");
  return SLD_OK;
}

sld_status batch_launch(sld_batch bt, float* ms) {
  cudaEventRecord(bt->ev0, bt->stream);
  cudaError_t e = cudaGraphLaunch(bt->plan.exec, bt->stream);
  cudaEventRecord(bt->ev1, bt->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(bt->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  cudaEventElapsedTime(ms, bt->ev0, bt->ev1);
  return SLD_OK;
}

}  // namespace

extern "C" {

sld_status sld_batch_create(sld_system* systems, int count, const sld_options* opt, sld_batch* out) {
  g_last_error.clear();
  if (!out) return fail(SLD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!systems || count < 1 || count > 4096) return fail(SLD_ERR_INVALID_ARG, "count must be in [1, 4096]");
  sld_options o;
  sld_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != SLD_FP64 && o.precision != SLD_FP32_IR)
    return fail(SLD_ERR_INVALID_ARG, "batched solves take SLD_FP64 or SLD_FP32_IR");
  if (!(o.tol > 0) || !(o.tol < 1) || !(o.inner_tol > 0) || !(o.inner_tol < 1) || !std::isfinite(o.fwd_tol) ||
      o.maxiter < 1 || o.max_outer < 1)
    return fail(SLD_ERR_INVALID_ARG, "bad tolerances or iteration caps");
  for (int k = 0; k < count; ++k) {
    sld_system s = systems[k];
    if (!s) return fail(SLD_ERR_INVALID_ARG, "a system is NULL");
    if (!s->deflation_ready) return fail(SLD_ERR_STATE, "every system needs sld_build_deflation first");
    if (s->kL > 0) return fail(SLD_ERR_INVALID_ARG, "extra dense deflation columns are not supported in a batched solve");
    if (s->device != systems[0]->device) return fail(SLD_ERR_INVALID_ARG, "systems on different devices");
    for (int j = 0; j < k; ++j)
      if (systems[j] == s) return fail(SLD_ERR_INVALID_ARG, "a system appears twice");
    sld_status st = ensure_workspace(s, o.precision == SLD_FP32_IR, false);
    if (st != SLD_OK) return st;
    cudaError_t e = cudaMemcpyAsync(s->bwork, s->b, sizeof(double) * s->g.n, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch rhs");
  }
  sld_batch bt = new sld_batch_s();
  bt->sys.assign(systems, systems + count);
  bt->o = o;
  cudaEventCreate(&bt->ev0);
  cudaEventCreate(&bt->ev1);
  {
    cudaError_t e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      sld_batch_destroy(bt);
      return cuda_fail(e, "batch stream");
    }
  }
  // candidate launch shapes: CTAs per SM, team-size exponent, cells per lane
  bool all4 = true;
  for (int k = 0; k < count; ++k) all4 = all4 && systems[k]->g.nx % 4 == 0 && systems[k]->g.nx >= 96;
  if (o.precision != SLD_FP64) all4 = false;  // the FP32-inner batch runs on the TMA sweeps (no cx choice)
  struct Cand { int per; double expo; int cx; };
  std::vector<Cand> cands;
  for (int cx : (all4 ? std::vector<int>{1, 4} : std::vector<int>{1}))
    cands.push_back({o.ctas_per_sm, 1.0, cx});
  if (o.ctas_per_sm > 0) cands = {{o.ctas_per_sm, 1.0, all4 ? 4 : 1}};
  // the trial solves also give the iterations of the measured-iterations plan
  const bool time_trials = cands.size() > 1 || o.ctas_per_sm <= 0;
  std::string times;
  float best_ms = 0.f;
  std::vector<double> last_teams(count, 1.0);  // the teams of the last timed launch
  for (size_t c = 0; c < cands.size(); ++c) {
    sld::BatchPlan trial;
    std::string msg;
    int st = sld::batch_build(bt->sys.data(), count, o, cands[c].per, cands[c].expo, nullptr, cands[c].cx, bt->stream,
                              &trial, &msg);
    if (st != SLD_OK) {
      sld::batch_free(&trial);
      if (cands.size() == 1 || c + 1 == cands.size()) {
        if (!bt->plan.exec) {
          sld_batch_destroy(bt);
          return fail((sld_status)st, msg);
        }
      }
      continue;
    }
    float ms = 0.f;
    if (time_trials) {  // time one full batched solve with this shape
      std::swap(bt->plan, trial);
      sld_status ls = batch_launch(bt, &ms);
      std::swap(bt->plan, trial);
      if (ls != SLD_OK) {
        sld::batch_free(&trial);
        sld_batch_destroy(bt);
        return ls;
      }
      times += " [cx " + std::to_string(cands[c].cx) + ", expo " + std::to_string(cands[c].expo).substr(0, 4) +
               ": " + std::to_string(ms).substr(0, 7) + " ms]";
    }
    for (int k = 0; k < count; ++k) last_teams[k] = trial.teams[k];
    if (!bt->plan.exec || ms < best_ms) {
      sld::batch_free(&bt->plan);
      bt->plan = trial;
      best_ms = ms;
    } else {
      sld::batch_free(&trial);
    }
  }
  // more candidates, teams rebalanced from measurement: each system's time
  // in the kernel (its team's first to last moment) in every timed launch
  // so far.  Where a system has been timed with two team sizes at least 25 %
  // apart, its time is modelled as a / t + b (b: the part more CTAs do not
  // shorten, such as its grid barriers), kept only if b is under 30 % of its
  // last time (the times are noisy, and a fit that calls most of the time
  // fixed starves the system of CTAs), else as proportional to 1 / t.  Up to
  // six rounds, ending after two that do not beat the best plan by 0.5 %;
  // the best is kept.
  std::vector<std::vector<std::pair<double, double>>> hist(count);  // (team size, ns) per timed launch
  auto record = [&]() {
    for (int k = 0; k < count; ++k) {
      double out[sld::kOutCount];
      if (cudaMemcpy(out, systems[k]->out, sizeof(out), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
      hist[k].push_back({last_teams[k], std::max(out[sld::kOutEndNs] - out[sld::kOutStartNs], 1.0)});
    }
    return true;
  };
  int stale = 0;
  for (int round = 0; round < 6 && stale < 2 && o.ctas_per_sm <= 0 && bt->plan.exec; ++round) {
    if (!record()) break;
    std::vector<double> ak(count), bk(count, 0.0);
    for (int k = 0; k < count; ++k) {
      const auto& h = hist[k];
      const auto last = h.back();
      ak[k] = last.second * last.first;  // proportional to 1 / t
      for (size_t i = h.size() - 1; i-- > 0;) {  // the latest earlier launch with another team size
        if (h[i].first == last.first) continue;
        if (std::fabs(h[i].first - last.first) < 0.25 * std::max(h[i].first, last.first)) break;
        const double u1 = 1.0 / last.first, u2 = 1.0 / h[i].first;
        const double a = (last.second - h[i].second) / (u1 - u2), b = last.second - a * u1;
        if (a > 0.0 && b >= 0.0 && b <= 0.3 * last.second) {
          ak[k] = a;
          bk[k] = b;
        }
        break;
      }
    }
    sld::BatchPlan trial;
    std::string msg;
    if (sld::batch_build(bt->sys.data(), count, o, bt->plan.per_sm, 1.0, ak.data(), bt->plan.cx, bt->stream, &trial,
                         &msg, bk.data()) != SLD_OK) {
      sld::batch_free(&trial);
      break;
    }
    float ms = 0.f;
    std::swap(bt->plan, trial);
    sld_status ls = batch_launch(bt, &ms);
    std::swap(bt->plan, trial);
    if (ls != SLD_OK) {
      sld::batch_free(&trial);
      sld_batch_destroy(bt);
      return ls;
    }
    times += " [rebalanced " + std::to_string(round + 1) + ": " + std::to_string(ms).substr(0, 7) + " ms]";
    for (int k = 0; k < count; ++k) last_teams[k] = trial.teams[k];
    stale = ms < 0.995f * best_ms ? 0 : stale + 1;
    if (ms < best_ms) {
      sld::batch_free(&bt->plan);
      bt->plan = trial;
      bt->plan.expo = -1.0;  // marks a rebalanced plan
      best_ms = ms;
    } else {
      sld::batch_free(&trial);
    }
  }
  const sld::BatchPlan& p = bt->plan;
  bt->desc = "systems " + std::to_string(count) + ", CTAs " + std::to_string(p.G) + " (" + std::to_string(p.per_sm) +
             " per SM), " + (p.tma ? std::string("TMA sweeps, 64x8 tiles") : "cells per lane " + std::to_string(p.cx)) +
             ", teams by " + (p.expo < 0 ? std::string("measured CTA-time") : "n^" + std::to_string(p.expo).substr(0, 4)) +
             ":";
  for (int k = 0; k < count; ++k) bt->desc += " " + std::to_string(p.teams[k]);
  if (!times.empty()) bt->desc += "; autotune:" + times;
  *out = bt;
  return SLD_OK;
}

sld_status sld_batch_solve(sld_batch bt, const double* const* b, double* const* x, sld_result* res) {
  g_last_error.clear();
  if (!bt) return fail(SLD_ERR_INVALID_ARG, "batch is NULL");
  const int count = (int)bt->sys.size();
  for (int k = 0; k < count; ++k) {
    sld_system s = bt->sys[k];
    const double* src = (b && b[k]) ? b[k] : s->b;
    cudaError_t e = cudaMemcpyAsync(s->bwork, src, sizeof(double) * s->g.n, kind_in(src), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch rhs");
  }
  float ms = 0.f;
  sld_status st = batch_launch(bt, &ms);
  if (st != SLD_OK) return st;
  sld_status worst = SLD_OK;
  std::string first_msg;
  for (int k = 0; k < count; ++k) {
    sld_result r{};
    sld_status sk = collect(bt->sys[k], bt->sys[k]->bwork, ms, x ? x[k] : nullptr, &r);
    if (res) res[k] = r;
    if (sk != SLD_OK && worst == SLD_OK) {
      worst = sk;
      first_msg = "system " + std::to_string(k) + ": " + g_last_error;
    }
  }
  // per-team span of the last launch, relative to the earliest team start
  {
    std::vector<double> t0(count), t1(count);
    bool ok = true;
    for (int k = 0; k < count && ok; ++k) {
      double out[sld::kOutCount];
      ok = cudaMemcpy(out, bt->sys[k]->out, sizeof(out), cudaMemcpyDeviceToHost) == cudaSuccess;
      t0[k] = out[sld::kOutStartNs];
      t1[k] = out[sld::kOutEndNs];
    }
    if (ok && count > 0) {
      const double base = *std::min_element(t0.begin(), t0.end());
      std::string d = bt->desc.substr(0, bt->desc.find("; last solve:"));
      d += "; last solve: team end ms:";
      char buf[32];
      for (int k = 0; k < count; ++k) {
        std::snprintf(buf, sizeof(buf), " %.1f", (t1[k] - base) * 1e-6);
        d += buf;
      }
      bt->desc = d;
    }
  }
  if (worst != SLD_OK) return fail(worst, first_msg);
  return SLD_OK;
}

const char* sld_batch_describe(sld_batch bt) { return bt ? bt->desc.c_str() : ""; }

void sld_batch_destroy(sld_batch bt) {
  if (!bt) return;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  sld::batch_free(&bt->plan);
  if (bt->stream) cudaStreamDestroy(bt->stream);
  if (bt->ev0) cudaEventDestroy(bt->ev0);
  if (bt->ev1) cudaEventDestroy(bt->ev1);
  delete bt;
}

sld_status sld_solve_batched(sld_system* systems, int count, const double* const* b, const sld_options* o,
                             double* const* x, sld_result* res) {
  sld_batch bt = nullptr;
  sld_status st = sld_batch_create(systems, count, o, &bt);
  if (st != SLD_OK) return st;
  st = sld_batch_solve(bt, b, x, res);
  sld_batch_destroy(bt);
  return st;
}

}  // extern "C"

namespace sld {
cudaError_t ensure_gacc(sld_system s, size_t doubles) {
  if (doubles <= s->gacc_cap && s->gacc) return cudaSuccess;
  if (s->gacc) {
    cudaStreamSynchronize(s->stream);
    cudaFree(s->gacc);
    s->gacc = nullptr;
    s->gacc_cap = 0;
  }
  cudaError_t e = cudaMalloc(&s->gacc, sizeof(double) * doubles);
  if (e == cudaSuccess) s->gacc_cap = doubles;
  return e;
}
}  // namespace sld

namespace sld {
cudaError_t ensure_gmres_ws(sld_system s, size_t doubles) {
  if (doubles <= s->gm_ws_cap && s->gm_ws) return cudaSuccess;
  if (s->gm_ws) {
    cudaStreamSynchronize(s->stream);
    cudaFree(s->gm_ws);
    s->gm_ws = nullptr;
    s->gm_ws_cap = 0;
  }
  cudaError_t e = cudaMalloc(&s->gm_ws, sizeof(double) * doubles);
  if (e == cudaSuccess) s->gm_ws_cap = doubles;
  return e;
}
}  // namespace sld
