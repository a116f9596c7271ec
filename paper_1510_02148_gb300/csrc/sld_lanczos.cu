// sld_lanczos.cu -- eigenpairs of the smallest nonzero eigenvalues of the
// label-deflated, Jacobi-preconditioned operator (the training targets of the
// deflation-vector network), by shift-invert Lanczos with full
// reorthogonalisation.
//
// Symmetric form: H = D^{-1/2} P A D^{-1/2}, P = I - A Z E^{-1} Z^T, D = diag A.
// P A is symmetric, so H is; H vanishes on span(D^{1/2} Z) and its other
// eigenvalues are those of M^{-1} P A (M = D), the spectrum deflated CG sees
// (Section 3.1).  The columns of D^{1/2} Z have disjoint supports (one label
// per cell), so projecting a vector off that span is a segmented sum.
//
// The smallest eigenvalues of H are small and clustered relative to its
// spread, so plain Lanczos needs thousands of steps for them.  Lanczos runs
// instead on S, the inverse of H on its range: for g in the range, with
// r = D^{1/2} g (then Z^T r = 0, so P r = r), t = A^{-1} r solves P A t = r,
// and S g = (D^{1/2} t projected onto the range).  The smallest eigenvalues
// lambda of H are the largest 1/lambda of S, well separated: a few tens of
// steps.  Each step is one solve with this library's deflated solver (FP32
// inner, FP64 refinement, relative residual 1e-10).  Lanczos vectors are
// FP64, reorthogonalised twice against all earlier ones; the tridiagonal
// matrix's largest eigenvalues come from Sturm-count bisection and its
// eigenvectors from inverse iteration, on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sld_net.h"
#include "sld_internal.h"

namespace {

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Start vector: SplitMix64 (Steele, Lea, Flood 2014) of the cell index,
// mapped to [-1, 1).
__global__ void k_start(int64_t n, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void k_scale(int64_t n, const double* __restrict__ a, const double* __restrict__ x,
                        double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] * x[i];
}

// out[label_i] += sqrt(D_i) h_i  (segmented sum, FP64 atomics)
__global__ void k_seg_sum(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ sq,
                          const double* __restrict__ h, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&out[label[i]], sq[i] * h[i]);
}

// h_i -= sqrt(D_i) c[label_i] / N[label_i]
__global__ void k_seg_remove(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ sq,
                             const double* __restrict__ c, const double* __restrict__ nrm, double* __restrict__ h) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int l = label[i];
    if (nrm[l] > 0.0) h[i] -= sq[i] * c[l] / nrm[l];
  }
}

// y = E^{-1} s, one warp per row
__global__ void k_gemv(int d, const double* __restrict__ M, const double* __restrict__ s, double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= d) return;
  double t = 0.0;
  for (int k = lane; k < d; k += 32) t += M[(int64_t)row * d + k] * s[k];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) y[row] = t;
}

__global__ void k_expand(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ y,
                         double* __restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = y[label[i]];
}

// w = dm * (u - u2)
__global__ void k_combine(int64_t n, const double* __restrict__ dm, const double* __restrict__ u,
                          const double* __restrict__ u2, double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = dm[i] * (u[i] - u2[i]);
}

// c[k] = V_k . w for k < nv (blockIdx.y = k), FP64 atomics of block sums
__global__ void k_multidot(int64_t n, const double* __restrict__ V, const double* __restrict__ w,
                           double* __restrict__ c) {
  __shared__ double red[8];
  const int k = blockIdx.y;
  const double* v = V + (int64_t)k * n;
  double t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t += v[i] * w[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) u += red[q];
    atomicAdd(&c[k], u);
  }
}

// w -= sum_{k < nv} c[k] V_k
__global__ void k_sub_comb(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ c,
                           double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = w[i];
  for (int k = 0; k < nv; ++k) t -= c[k] * V[(int64_t)k * n + i];
  w[i] = t;
}

// y = sum_{k < nv} c[k] V_k
__global__ void k_comb(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ c,
                       double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int k = 0; k < nv; ++k) t += c[k] * V[(int64_t)k * n + i];
  y[i] = t;
}

// y = a x + b y (y is not read when b == 0)
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

// out[i * k + j] = (float)(dm_i * y_i)
__global__ void k_store_vec(int64_t n, int k, int j, const double* __restrict__ dm, const double* __restrict__ y,
                            float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i * k + j] = (float)(dm[i] * y[i]);
}

__global__ void k_prep(int64_t n, const double* __restrict__ diag, double* __restrict__ dm, double* __restrict__ sq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    sq[i] = sqrt(diag[i]);
    dm[i] = 1.0 / sq[i];
  }
}

__global__ void k_seg_norm(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ diag,
                           double* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&nrm[label[i]], diag[i]);
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm).
int sturm(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    q = a[i] - x - (i ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Solve (T - s I) x = r for the tridiagonal T (a, b) by Gaussian elimination
// with partial pivoting (the band grows to two superdiagonals).
void tri_solve(const std::vector<double>& a, const std::vector<double>& b, double s, std::vector<double>& x) {
  const int m = (int)a.size();
  std::vector<double> d0(m), d1(m), d2(m);  // rows of U: diagonal, first and second superdiagonal
  std::vector<double> r = x;
  std::vector<double> dg(m), up(m), lo(m);
  for (int i = 0; i < m; ++i) {
    dg[i] = a[i] - s;
    up[i] = i + 1 < m ? b[i] : 0.0;
    lo[i] = i + 1 < m ? b[i] : 0.0;  // T[i+1][i]
  }
  // working row i: (u0 at col i, u1 at i+1, u2 at i+2)
  double u0 = dg[0], u1 = up[0], u2 = 0.0;
  for (int i = 0; i < m; ++i) {
    if (i + 1 < m) {
      // next row: (lo[i] at col i, dg[i+1] at i+1, up[i+1] at i+2)
      double n0 = lo[i], n1 = dg[i + 1], n2 = i + 2 < m ? up[i + 1] : 0.0;
      double rn = r[i + 1];
      if (std::fabs(n0) > std::fabs(u0)) {  // pivot: swap the rows
        std::swap(u0, n0);
        std::swap(u1, n1);
        std::swap(u2, n2);
        std::swap(r[i], rn);
      }
      if (u0 == 0.0) u0 = 1e-300;
      const double f = n0 / u0;
      d0[i] = u0;
      d1[i] = u1;
      d2[i] = u2;
      r[i + 1] = rn - f * r[i];
      u0 = n1 - f * u1;
      u1 = n2 - f * u2;
      u2 = 0.0;
    } else {
      d0[i] = u0 == 0.0 ? 1e-300 : u0;
      d1[i] = 0.0;
      d2[i] = 0.0;
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double t = r[i];
    if (i + 1 < m) t -= d1[i] * x[i + 1];
    if (i + 2 < m) t -= d2[i] * x[i + 2];
    x[i] = t / d0[i];
  }
}

}  // namespace

extern "C" sld_status sld_lanczos_eigvecs(sld_system s, int k, int m, double* vals, float* vecs, double* resid) {
  auto fail = [](sld_status st, const std::string& msg) {
    sld::set_last_error(msg);
    return st;
  };
  if (!s || !vals || !vecs) return fail(SLD_ERR_INVALID_ARG, "NULL argument");
  if (!s->deflation_ready || !s->label) return fail(SLD_ERR_STATE, "no deflation built");
  if (s->kL > 0) return fail(SLD_ERR_STATE, "build the label deflation alone (no extra columns) first");
  if (k < 1 || k > 8 || m <= k || m > 1000) return fail(SLD_ERR_INVALID_ARG, "need 1 <= k <= 8 and k < m <= 1000");
  const int64_t n = s->g.n;
  const int d = s->d;
  if (m > n) m = (int)n;
  cudaStream_t st = s->stream;
  double *V = nullptr, *work = nullptr;
  cudaError_t e = cudaMalloc(&V, sizeof(double) * (size_t)(m + 1) * n);
  if (e != cudaSuccess) return fail(SLD_ERR_OOM, "Lanczos basis: " + std::string(cudaGetErrorString(e)));
  // work: dm, sq, t, u, u2, w (n each), then seg (d), nrm (d), sv (d), yv (d), c (m+1)
  e = cudaMalloc(&work, sizeof(double) * ((size_t)6 * n + 4 * (size_t)d + m + 1));
  if (e != cudaSuccess) {
    cudaFree(V);
    return fail(SLD_ERR_OOM, "Lanczos work: " + std::string(cudaGetErrorString(e)));
  }
  double *dm = work, *sq = dm + n, *t = sq + n, *u = t + n, *u2 = u + n, *w = u2 + n;
  double *seg = w + n, *nrm = seg + d, *sv = nrm + d, *yv = sv + d, *c = yv + d;
  const unsigned B = nblk(n, 256);
  k_prep<<<B, 256, 0, st>>>(n, s->diag, dm, sq);
  cudaMemsetAsync(nrm, 0, sizeof(double) * d, st);
  k_seg_norm<<<B, 256, 0, st>>>(n, s->label, s->diag, nrm);
  auto project = [&](double* h) {  // h -= projection onto span(D^{1/2} Z)
    cudaMemsetAsync(seg, 0, sizeof(double) * d, st);
    k_seg_sum<<<B, 256, 0, st>>>(n, s->label, sq, h, seg);
    k_seg_remove<<<B, 256, 0, st>>>(n, s->label, sq, seg, nrm, h);
  };
  auto applyH = [&](const double* h, double* out) {
    k_scale<<<B, 256, 0, st>>>(n, dm, h, t);
    sld::launch_apply_A(s, t, u);
    sld::launch_restrict(s, u, sv);
    k_gemv<<<nblk(d, 4), 128, 0, st>>>(d, s->Einv, sv, yv);
    k_expand<<<B, 256, 0, st>>>(n, s->label, yv, t);
    sld::launch_apply_A(s, t, u2);
    k_combine<<<B, 256, 0, st>>>(n, dm, u, u2, out);
    project(out);
  };
  sld_options so;
  sld_default_options(&so);
  so.precision = SLD_FP32_IR;
  so.tol = 1e-10;
  sld_status solve_st = SLD_OK;
  auto applyS = [&](const double* h, double* out) {  // S h = range part of D^{1/2} A^{-1} D^{1/2} h
    k_scale<<<B, 256, 0, st>>>(n, sq, h, u);
    sld_result r{};
    const sld_status q = sld_solve(s, u, &so, t, &r);
    if (q != SLD_OK && q != SLD_ERR_NOT_CONVERGED) solve_st = q;
    k_scale<<<B, 256, 0, st>>>(n, sq, t, out);
    project(out);
  };
  const unsigned gd = std::min<unsigned>(B, 512);
  auto dot = [&](const double* a, const double* b2) -> double {  // via the multidot kernel, one vector
    cudaMemsetAsync(c, 0, sizeof(double), st);
    k_multidot<<<dim3(gd, 1), 256, 0, st>>>(n, a, b2, c);
    double h = 0.0;
    cudaMemcpyAsync(&h, c, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return h;
  };
  auto reorth = [&](int nv, double* x) {  // x -= V_{<nv} (V_{<nv}^T x), twice
    for (int pass = 0; pass < 2; ++pass) {
      cudaMemsetAsync(c, 0, sizeof(double) * nv, st);
      k_multidot<<<dim3(gd, nv), 256, 0, st>>>(n, V, x, c);
      k_sub_comb<<<B, 256, 0, st>>>(n, nv, V, c, x);
    }
  };
  std::vector<double> al, be;
  double* v0 = V;
  k_start<<<B, 256, 0, st>>>(n, v0);
  project(v0);
  double nv0 = std::sqrt(dot(v0, v0));
  if (!(nv0 > 0.0)) {
    cudaFree(V);
    cudaFree(work);
    return fail(SLD_ERR_BREAKDOWN, "start vector vanished");
  }
  k_axpby<<<B, 256, 0, st>>>(n, 1.0 / nv0, v0, 0.0, v0);
  int steps = 0;
  for (int j = 0; j < m; ++j) {
    double* vj = V + (int64_t)j * n;
    applyS(vj, w);
    if (solve_st != SLD_OK) break;
    const double a = dot(vj, w);
    k_axpby<<<B, 256, 0, st>>>(n, -a, vj, 1.0, w);
    if (j > 0) k_axpby<<<B, 256, 0, st>>>(n, -be.back(), V + (int64_t)(j - 1) * n, 1.0, w);
    reorth(j + 1, w);
    project(w);
    const double b2 = std::sqrt(dot(w, w));
    al.push_back(a);
    steps = j + 1;
    if (!(b2 > 1e-300) || j + 1 == m) {
      be.push_back(b2);
      break;
    }
    be.push_back(b2);
    k_axpby<<<B, 256, 0, st>>>(n, 1.0 / b2, w, 0.0, V + (int64_t)(j + 1) * n);
  }
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess || solve_st != SLD_OK) {
    cudaFree(V);
    cudaFree(work);
    if (solve_st != SLD_OK) return solve_st;  // sld_solve set the message
    return fail(SLD_ERR_CUDA, std::string("Lanczos: ") + cudaGetErrorString(e));
  }
  // Ritz pairs of the largest eigenvalues mu of T = tridiag(be, al, be);
  // lambda = 1 / mu
  const int mm = steps;
  std::vector<double> a(al.begin(), al.begin() + mm), b(be.begin(), be.begin() + std::max(0, mm - 1));
  double lo = a[0], hi = a[0];
  for (int i = 0; i < mm; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < mm ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const int kk = std::min(k, mm);
  std::vector<std::vector<double>> S;
  for (int j = 0; j < kk; ++j) {
    double l = lo, h = hi;
    const int idx = mm - 1 - j;  // j-th largest
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
      const double mid = 0.5 * (l + h);
      if (sturm(a, b, mid) > idx) h = mid;
      else l = mid;
    }
    const double theta = 0.5 * (l + h);
    vals[j] = 1.0 / theta;
    // inverse iteration, orthogonalised against the earlier vectors
    std::vector<double> x(mm);
    for (int i = 0; i < mm; ++i) x[i] = 1.0 + 0.01 * std::sin(1.0 + 7.0 * i + 3.0 * j);
    const double shift = theta - 1e-12 * std::max(1.0, std::fabs(theta));
    for (int it = 0; it < 4; ++it) {
      tri_solve(a, b, shift, x);
      for (const auto& q : S) {
        double p = 0.0;
        for (int i = 0; i < mm; ++i) p += q[i] * x[i];
        for (int i = 0; i < mm; ++i) x[i] -= p * q[i];
      }
      double nn = 0.0;
      for (double v : x) nn += v * v;
      nn = std::sqrt(nn);
      for (double& v : x) v /= nn;
    }
    S.push_back(x);
  }
  // Ritz vectors h_j = V s_j, output v_j = D^{-1/2} h_j
  float* out = vecs;
  float* staged = nullptr;
  cudaPointerAttributes at;
  const bool dev = cudaPointerGetAttributes(&at, vecs) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (!dev) {
    e = cudaMalloc(&staged, sizeof(float) * (size_t)n * k);
    if (e != cudaSuccess) {
      cudaFree(V);
      cudaFree(work);
      return fail(SLD_ERR_OOM, "Lanczos output staging");
    }
    out = staged;
  }
  cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n * k, st);
  for (int j = 0; j < kk; ++j) {
    cudaMemcpyAsync(c, S[j].data(), sizeof(double) * mm, cudaMemcpyHostToDevice, st);
    k_comb<<<B, 256, 0, st>>>(n, mm, V, c, w);
    k_store_vec<<<B, 256, 0, st>>>(n, k, j, dm, w, out);
    if (resid) {  // ||H h - lambda h||_2, ||h|| = 1
      applyH(w, t);
      k_axpby<<<B, 256, 0, st>>>(n, -vals[j], w, 1.0, t);
      resid[j] = std::sqrt(dot(t, t));
    }
  }
  if (!dev) e = cudaMemcpyAsync(vecs, out, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (staged) cudaFree(staged);
  cudaFree(V);
  cudaFree(work);
  if (e != cudaSuccess) return fail(SLD_ERR_CUDA, std::string("Lanczos vectors: ") + cudaGetErrorString(e));
  for (int j = kk; j < k; ++j) vals[j] = NAN;
  return SLD_OK;
}
