// FP64 vector kernels of the Davidson eigensolver (the diagonalisation of
// Sec. II): deterministic two-stage reductions (per-CTA partials summed in
// a fixed order), subspace combinations, preconditioner, and a one-CTA
// cyclic Jacobi eigensolver for the projected matrix (at most 32 x 32).
#include <cuda_runtime.h>

#include <cstdint>

namespace su2 {
namespace {

constexpr int kMaxSub = 32;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial[blockIdx.x * nvec + i] = sum over this CTA's slice of V_i . w
__global__ void __launch_bounds__(kRedThreads) multidot_kernel(const double* __restrict__ V, int64_t ldv, int nvec,
                                                               const double* __restrict__ w, int64_t n,
                                                               double* __restrict__ partial, const int* __restrict__ dn) {
  if (dn) nvec = *dn + nvec;
  __shared__ double red[kRedThreads / 32][kMaxSub];
  double acc[kMaxSub];
#pragma unroll
  for (int i = 0; i < kMaxSub; ++i) acc[i] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride) {
    const double wx = w[x];
#pragma unroll
    for (int i = 0; i < kMaxSub; ++i)
      if (i < nvec) acc[i] = fma(V[i * ldv + x], wx, acc[i]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kMaxSub; ++i) {
    if (i >= nvec) break;
    const double s = warp_sum(acc[i]);
    if (lane == 0) red[wid][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double s = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) s += red[q][threadIdx.x];
    partial[int64_t(blockIdx.x) * nvec + threadIdx.x] = s;
  }
}

// out[i] = scale * sum_g partial[g*nvec + i]  (fixed order)
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int ng, int nvec, double scale,
                                       double* __restrict__ out, const int* __restrict__ dn) {
  if (dn) nvec = *dn + nvec;
  const int i = threadIdx.x;
  if (i < nvec) {
    double s = 0.0;
    for (int g = 0; g < ng; ++g) s += partial[int64_t(g) * nvec + i];
    out[i] = scale * s;
  }
}

// out = sum_i y[i] V_i    (and optionally out2 = sum_i y[i] W_i)
__global__ void combine_kernel(const double* __restrict__ V, const double* __restrict__ W, int64_t ldv, int nvec,
                               const double* __restrict__ y, int64_t n, double* __restrict__ out,
                               double* __restrict__ out2, const int* __restrict__ dn) {
  if (dn) nvec = *dn + nvec;
  __shared__ double sy[kMaxSub];
  if (threadIdx.x < nvec) sy[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nvec; ++i) {
      a = fma(sy[i], V[i * ldv + x], a);
      if (W) b = fma(sy[i], W[i * ldv + x], b);
    }
    out[x] = a;
    if (W) out2[x] = b;
  }
}

// t -= sum_i h[i] V_i
__global__ void subtract_kernel(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                                int64_t n, double* __restrict__ t, const int* __restrict__ dn) {
  if (dn) nvec = *dn + nvec;
  __shared__ double sh[kMaxSub];
  if (threadIdx.x < nvec) sh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride) {
    double a = t[x];
    for (int i = 0; i < nvec; ++i) a = fma(-sh[i], V[i * ldv + x], a);
    t[x] = a;
  }
}

// r = ax - theta x
__global__ void residual_kernel(const double* __restrict__ x, const double* __restrict__ ax,
                                const double* __restrict__ theta, int64_t n, double* __restrict__ r) {
  const double th = *theta;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) r[i] = fma(-th, x[i], ax[i]);
}

// t = r / (diag - theta), |diag - theta| clamped to >= 1e-12 (sign kept)
__global__ void precond_kernel(const double* __restrict__ r, const double* __restrict__ diag,
                               const double* __restrict__ theta, int64_t n, double* __restrict__ t) {
  const double th = *theta;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = diag[i] - th;
    if (fabs(d) < 1e-12) d = d >= 0.0 ? 1e-12 : -1e-12;
    t[i] = r[i] / d;
  }
}

// y = x * s[0]^(-1/2) when s holds a squared norm
__global__ void scale_kernel(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ nrm2,
                             int64_t n) {
  const double s = 1.0 / sqrt(*nrm2);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = x[i] * s;
}

// cyclic Jacobi on the symmetrised nsub x nsub matrix H (leading dim ld);
// outputs ascending eigenvalues w and eigenvectors Y (column j, ld rows)
__global__ void jacobi_kernel(const double* __restrict__ H, int ld, int n, double* __restrict__ w,
                              double* __restrict__ Y, int* __restrict__ status, const int* __restrict__ dn) {
  if (dn) n = *dn + n;
  __shared__ double A[kMaxSub][kMaxSub + 1], V[kMaxSub][kMaxSub + 1];
  __shared__ double cs[2];
  __shared__ int done;
  const int t = threadIdx.x;
  for (int idx = t; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, j = idx / n;
    A[i][j] = 0.5 * (H[i + j * ld] + H[j + i * ld]);
    V[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (t == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          tot += A[i][j] * A[i][j];
          if (i != j) off += A[i][j] * A[i][j];
        }
      done = (off <= 1e-30 * tot) || tot == 0.0;
    }
    __syncthreads();
    if (done) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (t == 0) {
          const double apq = A[p][q];
          double c = 1.0, s = 0.0;
          if (apq != 0.0) {
            const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          if (t < n) {  // columns p, q
            const double akp = A[t][p], akq = A[t][q];
            A[t][p] = c * akp - s * akq;
            A[t][q] = s * akp + c * akq;
            const double vkp = V[t][p], vkq = V[t][q];
            V[t][p] = c * vkp - s * vkq;
            V[t][q] = s * vkp + c * vkq;
          }
          __syncthreads();
          if (t < n) {  // rows p, q
            const double apk = A[p][t], aqk = A[q][t];
            A[p][t] = c * apk - s * aqk;
            A[q][t] = s * apk + c * aqk;
          }
        }
        __syncthreads();
      }
  }
  if (t == 0) {
    // selection sort of eigenpairs, ascending
    int order[kMaxSub];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (A[order[j]][order[j]] < A[order[i]][order[i]]) {
          const int tmp = order[i];
          order[i] = order[j];
          order[j] = tmp;
        }
    for (int j = 0; j < n; ++j) {
      w[j] = A[order[j]][order[j]];
      for (int i = 0; i < n; ++i) Y[i + j * ld] = V[i][order[j]];
    }
    if (!done) *status = 4;
  }
}

// partial max |x| and its index per CTA
__global__ void absmax_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ pv,
                              int64_t* __restrict__ pi) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double best = -1.0;
  int64_t bi = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = fabs(x[i]);
    if (a > best) { best = a; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = sv[threadIdx.x + o];
      const int64_t ai = si[threadIdx.x + o];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && ai < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

__global__ void diag_set_kernel(double* __restrict__ H, int ld, int n, const double* __restrict__ w) {
  for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
    const int i = idx % ld, j = idx / ld;
    H[idx] = (i == j && i < n) ? w[i] : 0.0;
  }
}

__global__ void copy_col_kernel(double* __restrict__ H, int ld, int col, const double* __restrict__ h, int n,
                                const int* __restrict__ dn) {
  if (dn) {  // column nsub-1, n = nsub
    n = *dn;
    col = n - 1;
  }
  const int i = threadIdx.x;
  if (i < n) {
    H[i + col * ld] = h[i];
    H[col + i * ld] = h[i];
  }
}

// ---- device-side subspace bookkeeping (graph-capturable Davidson iteration)
// dst = V[nsub-1] (dir 0) or V[nsub-1] = src (dir 1)
__global__ void newest_copy_kernel(double* __restrict__ V, int64_t n, const int* __restrict__ dn,
                                   double* __restrict__ w, int dir) {
  const int64_t base = int64_t(*dn - 1) * n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (dir == 0) w[i] = V[base + i];
    else V[base + i] = w[i];
  }
}

// restart when the subspace is full: V[q] <- V Y[:, q], AV[q] <- AV Y[:, q]
// for q < keep (into tmp, then back), H <- diag(w[:keep]); sets *dn = keep
__global__ void restart_combine_kernel(const double* __restrict__ V, const double* __restrict__ AV, int64_t n,
                                       const double* __restrict__ Y, int ld, int keep, int max_sub,
                                       const int* __restrict__ dn, double* __restrict__ tmp) {
  if (*dn < max_sub) return;
  const int nv = *dn;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride)
    for (int q = 0; q < keep; ++q) {
      double a = 0.0, b = 0.0;
      for (int i = 0; i < nv; ++i) {
        a = fma(Y[i + q * ld], V[int64_t(i) * n + x], a);
        b = fma(Y[i + q * ld], AV[int64_t(i) * n + x], b);
      }
      tmp[int64_t(2 * q) * n + x] = a;
      tmp[int64_t(2 * q + 1) * n + x] = b;
    }
}
__global__ void restart_copy_kernel(double* __restrict__ V, double* __restrict__ AV, int64_t n, int keep, int max_sub,
                                    const int* __restrict__ dn, const double* __restrict__ tmp) {
  if (*dn < max_sub) return;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride)
    for (int q = 0; q < keep; ++q) {
      V[int64_t(q) * n + x] = tmp[int64_t(2 * q) * n + x];
      AV[int64_t(q) * n + x] = tmp[int64_t(2 * q + 1) * n + x];
    }
}
__global__ void restart_finish_kernel(double* __restrict__ H, int ld, const double* __restrict__ w, int keep,
                                      int max_sub, int* __restrict__ dn) {
  if (*dn < max_sub) return;
  __syncthreads();
  for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
    const int i = idx % ld, j = idx / ld;
    H[idx] = (i == j && i < keep) ? w[i] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *dn = keep;
}
// V[nsub] = t / ||t|| when ||t||^2 > tiny (else the subspace is left as is)
__global__ void append_kernel(double* __restrict__ V, int64_t n, const int* __restrict__ dn,
                              const double* __restrict__ t, const double* __restrict__ nrm2) {
  if (!(*nrm2 > 1e-28)) return;
  const double s = 1.0 / sqrt(*nrm2);
  const int64_t base = int64_t(*dn) * n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) V[base + i] = t[i] * s;
}
__global__ void append_count_kernel(int* __restrict__ dn, const double* __restrict__ nrm2) {
  if (threadIdx.x == 0 && *nrm2 > 1e-28) *dn += 1;
}

}  // namespace

int dav_grid(int64_t n) {
  int g = int((n + 255) / 256);
  return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
}

void dav_multidot(cudaStream_t s, const double* V, int64_t ldv, int nvec, const double* w, int64_t n,
                  double* partial, double* out, double scale, const int* dn) {
  const int g = dav_grid(n);
  multidot_kernel<<<g, kRedThreads, 0, s>>>(V, ldv, nvec, w, n, partial, dn);
  reduce_partials_kernel<<<1, 32, 0, s>>>(partial, g, nvec, scale, out, dn);
}
void dav_combine(cudaStream_t s, const double* V, const double* W, int64_t ldv, int nvec, const double* y, int64_t n,
                 double* out, double* out2, const int* dn) {
  combine_kernel<<<dav_grid(n), 256, 0, s>>>(V, W, ldv, nvec, y, n, out, out2, dn);
}
void dav_subtract(cudaStream_t s, const double* V, int64_t ldv, int nvec, const double* h, int64_t n, double* t,
                  const int* dn) {
  subtract_kernel<<<dav_grid(n), 256, 0, s>>>(V, ldv, nvec, h, n, t, dn);
}
void dav_residual(cudaStream_t s, const double* x, const double* ax, const double* theta, int64_t n, double* r) {
  residual_kernel<<<dav_grid(n), 256, 0, s>>>(x, ax, theta, n, r);
}
void dav_precond(cudaStream_t s, const double* r, const double* diag, const double* theta, int64_t n, double* t) {
  precond_kernel<<<dav_grid(n), 256, 0, s>>>(r, diag, theta, n, t);
}
void dav_scale(cudaStream_t s, double* y, const double* x, const double* nrm2, int64_t n) {
  scale_kernel<<<dav_grid(n), 256, 0, s>>>(y, x, nrm2, n);
}
void dav_jacobi(cudaStream_t s, const double* H, int ld, int n, double* w, double* Y, int* status, const int* dn) {
  jacobi_kernel<<<1, 32, 0, s>>>(H, ld, n, w, Y, status, dn);
}
void dav_absmax(cudaStream_t s, const double* x, int64_t n, double* pv, int64_t* pi, int* ng) {
  const int g = dav_grid(n);
  *ng = g;
  absmax_kernel<<<g, 256, 0, s>>>(x, n, pv, pi);
}
void dav_diag_set(cudaStream_t s, double* H, int ld, int n, const double* w) {
  diag_set_kernel<<<1, 256, 0, s>>>(H, ld, n, w);
}
void dav_copy_col(cudaStream_t s, double* H, int ld, int col, const double* h, int n, const int* dn) {
  copy_col_kernel<<<1, 32, 0, s>>>(H, ld, col, h, n, dn);
}
void dav_newest(cudaStream_t s, double* V, int64_t n, const int* dn, double* w, int dir) {
  newest_copy_kernel<<<dav_grid(n), 256, 0, s>>>(V, n, dn, w, dir);
}
void dav_restart(cudaStream_t s, double* V, double* AV, int64_t n, const double* Y, int ld, double* H,
                 const double* w, int keep, int max_sub, int* dn, double* tmp) {
  restart_combine_kernel<<<dav_grid(n), 256, 0, s>>>(V, AV, n, Y, ld, keep, max_sub, dn, tmp);
  restart_copy_kernel<<<dav_grid(n), 256, 0, s>>>(V, AV, n, keep, max_sub, dn, tmp);
  restart_finish_kernel<<<1, 256, 0, s>>>(H, ld, w, keep, max_sub, dn);
}
void dav_append(cudaStream_t s, double* V, int64_t n, int* dn, const double* t, const double* nrm2) {
  append_kernel<<<dav_grid(n), 256, 0, s>>>(V, n, dn, t, nrm2);
  append_count_kernel<<<1, 32, 0, s>>>(dn, nrm2);
}

}  // namespace su2
