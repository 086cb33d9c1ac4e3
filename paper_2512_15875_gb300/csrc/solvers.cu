// Solver drivers on the GPU (Sec. II.B-C): QR gauge moves of the orthogonality centre, an
// on-demand environment cache, batched MINRES (Paige & Saunders 1975) with device-side Lanczos
// and Givens scalars, ALS and variational-fitting sweeps, Rayleigh-Ritz in float64 (cyclic
// Jacobi), and block LOBPCG (Alg. 2).
//
// Readings of points the paper leaves open (same as the oracle): the solution TTNS is kept in
// canonical form with the centre at the node being updated (R with a non-negative diagonal);
// sweeps visit the nodes in depth-first pre-order from the root; MINRES warm-starts from the
// current node tensor; fitting starts from the input state of the largest |coefficient|;
// LOBPCG updates x_j = sum_{k<=3n} v_kj s_k (normalised), p_j = sum_{k>n} v_kj s_k and uses
// S = {x} u {r} in its first iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

ttn_ttno* identity_for(ttn_ctx* ctx, const TreeInfo& tree);
template <class T>
void gram_pairs(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                const std::vector<int>& pb, const std::vector<int>& pk, double* d_out);
unsigned gram_device(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                     double* d_mat, int ld, int prec);

namespace {

constexpr int kT = 256;

int grid_of(long long n) {
  long long b = (n + kT - 1) / kT;
  return (int)std::max<long long>(1, std::min<long long>(b, 152 * 32));
}

// ----------------------------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------------------------

template <class T>
__device__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Householder QR of one rows x D matrix per CTA (row-major, rows >= D): the reflectors
// overwrite the working copy of A, Q (rows x D) and R (D x D, non-negative diagonal) are written
// out. With in_smem the working copies of A and Q live in dynamic shared memory (2 rows D
// elements), so the column passes read and write on chip; A in global memory is then left as
// it was.
template <class T>
__global__ void __launch_bounds__(kT) householder_qr_kernel(T* __restrict__ A_g,
                                                           T* __restrict__ Q_g,
                                                           T* __restrict__ R, int rows, int D,
                                                           long long mstride, int in_smem) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  T* A = A_g + (long long)blockIdx.x * mstride;
  T* Q = Q_g + (long long)blockIdx.x * mstride;
  T* const Q_out = Q;
  if (in_smem) {
    T* As = reinterpret_cast<T*>(qr_smem);
    for (long long i = threadIdx.x; i < (long long)rows * D; i += blockDim.x) As[i] = A[i];
    A = As;
    Q = As + (long long)rows * D;
    __syncthreads();
  }
  R += (long long)blockIdx.x * D * D;
  __shared__ T red[33];
  __shared__ T tau[64];
  __shared__ T wk[8][32];
  __shared__ T par[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < D; ++j) {
    T part = 0;
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) {
      const T x = A[(long long)i * D + j];
      part += x * x;
    }
    const T sigma = block_sum(part, red);
    if (threadIdx.x == 0) {
      const T alpha = A[(long long)j * D + j];
      if (sigma == T(0)) {
        tau[j] = 0;
        par[0] = 0;
      } else {
        const T normx = sqrt(alpha * alpha + sigma);
        const T beta = alpha <= T(0) ? normx : -normx;
        tau[j] = (beta - alpha) / beta;
        par[0] = T(1) / (alpha - beta);
        A[(long long)j * D + j] = beta;
      }
    }
    __syncthreads();
    const T tj = tau[j];
    if (tj != T(0)) {
      const T sc = par[0];
      for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) A[(long long)i * D + j] *= sc;
      __syncthreads();
      for (int k0 = j + 1; k0 < D; k0 += 32) {
        const int k = k0 + lane;
        T acc = 0;
        if (k < D)
          for (int i = j + warp; i < rows; i += 8) {
            const T v = i == j ? T(1) : A[(long long)i * D + j];
            acc += v * A[(long long)i * D + k];
          }
        wk[warp][lane] = acc;
        __syncthreads();
        T w = 0;
        for (int q = 0; q < 8; ++q) w += wk[q][lane];
        __syncthreads();
        if (k < D)
          for (int i = j + warp; i < rows; i += 8) {
            const T v = i == j ? T(1) : A[(long long)i * D + j];
            A[(long long)i * D + k] -= tj * v * w;
          }
        __syncthreads();
      }
    }
  }
  for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
    const int a = idx / D, b = idx % D;
    R[idx] = b >= a ? A[(long long)a * D + b] : T(0);
  }
  for (long long idx = threadIdx.x; idx < (long long)rows * D; idx += blockDim.x) {
    const long long i = idx / D;
    const int k = (int)(idx % D);
    Q[idx] = i == k ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = D - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == T(0)) continue;
    for (int k0 = j; k0 < D; k0 += 32) {
      const int k = k0 + lane;
      T acc = 0;
      if (k < D)
        for (int i = j + warp; i < rows; i += 8) {
          const T v = i == j ? T(1) : A[(long long)i * D + j];
          acc += v * Q[(long long)i * D + k];
        }
      wk[warp][lane] = acc;
      __syncthreads();
      T w = 0;
      for (int q = 0; q < 8; ++q) w += wk[q][lane];
      __syncthreads();
      if (k < D)
        for (int i = j + warp; i < rows; i += 8) {
          const T v = i == j ? T(1) : A[(long long)i * D + j];
          Q[(long long)i * D + k] -= tj * v * w;
        }
      __syncthreads();
    }
  }
  // sign convention: diag(R) >= 0
  for (int j = 0; j < D; ++j) {
    if (R[j * D + j] < T(0)) {
      __syncthreads();
      for (int b = j + threadIdx.x; b < D; b += blockDim.x) R[j * D + b] = -R[j * D + b];
      for (int i = threadIdx.x; i < rows; i += blockDim.x) Q[(long long)i * D + j] =
          -Q[(long long)i * D + j];
    }
    __syncthreads();
  }
  if (in_smem) {
    __syncthreads();
    for (long long i = threadIdx.x; i < (long long)rows * D; i += blockDim.x) Q_out[i] = Q[i];
  }
}

// out[s][o][k][i] = sum_b R[s][k][b] in[s][o][b][i]
template <class T>
__global__ void leg_product_kernel(const T* __restrict__ R, const T* __restrict__ in,
                                   T* __restrict__ out, int n, long long size, long long inner,
                                   int D) {
  const long long total = (long long)n * size;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long s = idx / size;
    const long long r = idx - s * size;
    const long long i = r % inner;
    const long long k = (r / inner) % D;
    const long long o = r / (inner * D);
    const T* Rk = R + (s * D + k) * D;
    const T* src = in + s * size + o * D * inner + i;
    T acc = 0;
    for (int b = 0; b < D; ++b) acc += Rk[b] * src[(long long)b * inner];
    out[idx] = acc;
  }
}

// out[s] = sum_i x[s][i] * y[s][i] in float64, one CTA per state
template <class T>
__global__ void dot_kernel(const T* __restrict__ x, const T* __restrict__ y, long long n,
                           double* __restrict__ out) {
  __shared__ double red[33];
  const long long off = (long long)blockIdx.x * n;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x)
    acc += (double)x[off + i] * (double)y[off + i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

template <class T>
__global__ void scale_kernel(T* __restrict__ x, const double* __restrict__ f, long long n,
                             int mode, int n_states) {
  // mode 0: x *= f[s]; mode 1: x *= 1/sqrt(f[s]) (f > 0)
  const long long total = (long long)n * n_states;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const double g = f[idx / n];
    const double sc = mode == 0 ? g : (g > 0.0 ? 1.0 / sqrt(g) : 0.0);
    x[idx] = (T)((double)x[idx] * sc);
  }
}

// out[j][i] (+)= sum_{p in [seg[j], seg[j+1])} coef[p] * Y[p][i]
template <class T>
__global__ void seg_sum_kernel(const T* __restrict__ Y, const int* __restrict__ seg,
                               const double* __restrict__ coef, T* __restrict__ out, int n_out,
                               long long size, int accumulate) {
  const long long total = (long long)n_out * size;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / size);
    const long long i = idx - (long long)j * size;
    T acc = accumulate ? out[idx] : T(0);
    for (int p = seg[j]; p < seg[j + 1]; ++p) acc += (T)coef[p] * Y[(long long)p * size + i];
    out[idx] = acc;
  }
}

// ---- MINRES (batched over states; scalars in float64) ----------------------------------------
enum { MR_BETA1, MR_BNORM, MR_BETA, MR_C1, MR_S1, MR_C2, MR_S2, MR_PHIBAR, MR_ACTIVE, MR_ALPHA,
       MR_BNEXT2, MR_DELTA, MR_EPS, MR_GAMMA, MR_TAU, MR_BNEXT, MR_UPD, MR_CONT, MR_ITS,
       MR_HITCAP, MR_TNORM2, MR_NFIELDS };

__global__ void mr_init_scalars(double* sc, const double* bb, const double* rr, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double* f = sc + (long long)s * MR_NFIELDS;
  const double beta1 = sqrt(fmax(rr[s], 0.0)), bnorm = sqrt(fmax(bb[s], 0.0));
  f[MR_BETA1] = beta1;
  f[MR_BNORM] = bnorm;
  f[MR_BETA] = beta1;
  f[MR_C1] = 1.0;
  f[MR_S1] = 0.0;
  f[MR_C2] = 1.0;
  f[MR_S2] = 0.0;
  f[MR_PHIBAR] = beta1;
  f[MR_ACTIVE] = (beta1 > 0.0 && bnorm > 0.0) ? 1.0 : 0.0;
  f[MR_ITS] = 0.0;
  f[MR_HITCAP] = 0.0;
  f[MR_TNORM2] = 0.0;
}

// r = b - Ax (in p), v = r / beta1, vp = 0, w1 = w2 = 0
template <class T>
__global__ void mr_init_vectors(const double* sc, const T* b, const T* Ax, T* v, T* vp, T* w1,
                                T* w2, long long n, int n_states) {
  const long long total = n * n_states;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const double* f = sc + (idx / n) * MR_NFIELDS;
    const double beta1 = f[MR_BETA1];
    const T r = b[idx] - Ax[idx];
    v[idx] = beta1 > 0.0 ? (T)((double)r / beta1) : T(0);
    vp[idx] = T(0);
    w1[idx] = T(0);
    w2[idx] = T(0);
  }
}

// r = b - Ax stored into Ax's buffer (for the initial residual norm)
template <class T>
__global__ void sub_kernel(const T* b, T* Ax, long long total) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    Ax[idx] = b[idx] - Ax[idx];
}

// p = p - alpha v - beta vp
template <class T>
__global__ void mr_lanczos(const double* sc, const double* alpha, T* p, const T* v, const T* vp,
                           long long n, int n_states) {
  const long long total = n * n_states;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long s = idx / n;
    const double* f = sc + s * MR_NFIELDS;
    p[idx] = (T)((double)p[idx] - alpha[s] * (double)v[idx] - f[MR_BETA] * (double)vp[idx]);
  }
}

__global__ void mr_step_scalars(double* sc, const double* alpha, const double* bnext2, int n,
                                double tol, int maxiter) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double* f = sc + (long long)s * MR_NFIELDS;
  f[MR_UPD] = 0.0;
  f[MR_CONT] = 0.0;
  if (f[MR_ACTIVE] == 0.0) return;
  const double a = alpha[s], beta = f[MR_BETA];
  const double bnext = sqrt(fmax(bnext2[s], 0.0));
  f[MR_TNORM2] += a * a + beta * beta + bnext * bnext;
  const double eps = f[MR_S2] * beta;
  const double dtil = f[MR_C2] * beta;
  const double delta = f[MR_C1] * dtil + f[MR_S1] * a;
  const double gtil = -f[MR_S1] * dtil + f[MR_C1] * a;
  const double gamma = hypot(gtil, bnext);
  f[MR_ITS] += 1.0;
  if (gamma == 0.0) {
    f[MR_ACTIVE] = 0.0;
    return;
  }
  const double c = gtil / gamma, sn = bnext / gamma;
  const double tau = c * f[MR_PHIBAR];
  f[MR_PHIBAR] = -sn * f[MR_PHIBAR];
  f[MR_DELTA] = delta;
  f[MR_EPS] = eps;
  f[MR_GAMMA] = gamma;
  f[MR_TAU] = tau;
  f[MR_BNEXT] = bnext;
  f[MR_C2] = f[MR_C1];
  f[MR_S2] = f[MR_S1];
  f[MR_C1] = c;
  f[MR_S1] = sn;
  f[MR_UPD] = 1.0;
  const bool conv = bnext == 0.0 || fabs(f[MR_PHIBAR]) <= tol * f[MR_BNORM];
  f[MR_CONT] = conv ? 0.0 : 1.0;
  f[MR_ACTIVE] = conv ? 0.0 : 1.0;
  if (!conv && f[MR_ITS] >= maxiter) f[MR_HITCAP] = 1.0;
  f[MR_BETA] = bnext;
}

// Paige-Saunders stop on the rounding level of the iterate: a state that is still running stops
// once |phibar_k| <= eps_T * (|T_k|_F |x_k| + |b|) (|x_k|^2 in xx, eps_T the machine epsilon
// of the vector type). Beyond it the recurrence residual no longer describes x_k; this is what a
// Rayleigh-quotient shift that has converged to working precision runs into (Alg. 3).
__global__ void mr_floor_check(double* sc, const double* xx, int n, double eps) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double* f = sc + (long long)s * MR_NFIELDS;
  if (f[MR_UPD] == 0.0 || f[MR_CONT] == 0.0) return;
  const double floor_r = eps * (sqrt(f[MR_TNORM2]) * sqrt(fmax(xx[s], 0.0)) + f[MR_BNORM]);
  if (fabs(f[MR_PHIBAR]) <= floor_r) {
    f[MR_CONT] = 0.0;
    f[MR_ACTIVE] = 0.0;
    f[MR_HITCAP] = 0.0;
  }
}

template <class T>
__global__ void mr_step_vectors(const double* sc, T* x, T* v, T* vp, T* w1, T* w2, const T* p,
                                long long n, int n_states) {
  const long long total = n * n_states;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const double* f = sc + (idx / n) * MR_NFIELDS;
    if (f[MR_UPD] == 0.0) continue;
    const double wn = ((double)v[idx] - f[MR_DELTA] * (double)w1[idx] -
                       f[MR_EPS] * (double)w2[idx]) / f[MR_GAMMA];
    x[idx] = (T)((double)x[idx] + f[MR_TAU] * wn);
    w2[idx] = w1[idx];
    w1[idx] = (T)wn;
    if (f[MR_CONT] != 0.0) {
      vp[idx] = v[idx];
      v[idx] = (T)((double)p[idx] / f[MR_BNEXT]);
    }
  }
}

// ---- Rayleigh-Ritz: cyclic Jacobi (round-robin parallel ordering), one CTA, float64 ---------
// off_out (may be NULL) receives sqrt(off-diagonal / total) of A's squared entries when the
// kernel returns: at most tol when it stopped on the tolerance, the reached value after
// max_sweeps otherwise.
__global__ void __launch_bounds__(1024) jacobi_kernel(double* A, double* V, int m, int max_sweeps,
                                                      double tol, double* off_out) {
  extern __shared__ double sh[];
  const int mp = m + (m & 1);
  const int npairs = mp / 2;
  double* cs = sh;              // npairs
  double* sn = sh + npairs;     // npairs
  int* pp = reinterpret_cast<int*>(sh + 2 * npairs);
  int* qq = pp + npairs;
  __shared__ double red[33];
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x)
    V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const double a = A[idx];
      tot += a * a;
      if (idx / m != idx % m) off += a * a;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    const bool done = off <= tol * tol * tot;
    if (done || sweep == max_sweeps) {
      if (off_out && threadIdx.x == 0) off_out[0] = tot > 0.0 ? sqrt(off / tot) : 0.0;
      break;
    }
    for (int r = 0; r < mp - 1; ++r) {
      for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = 0;
          q = (r % (mp - 1)) + 1;
        } else {
          p = ((i + r) % (mp - 1)) + 1;
          q = ((mp - 1 - i + r) % (mp - 1)) + 1;
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        pp[i] = p;
        qq[i] = q;
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * m + q];
          if (apq != 0.0) {
            const double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = threadIdx.x; idx < npairs * m; idx += blockDim.x) {
        const int i = idx / m, j = idx % m;
        const int p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = A[p * m + j], aq = A[q * m + j];
        A[p * m + j] = c * ap - s * aq;
        A[q * m + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = threadIdx.x; idx < npairs * m; idx += blockDim.x) {
        const int i = idx / m, j = idx % m;
        const int p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = A[j * m + p], aq = A[j * m + q];
        A[j * m + p] = c * ap - s * aq;
        A[j * m + q] = s * ap + c * aq;
        const double vp = V[j * m + p], vq = V[j * m + q];
        V[j * m + p] = c * vp - s * vq;
        V[j * m + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// Cyclic Jacobi across the whole grid (cooperative launch; all CTAs resident). Each round of the
// round-robin ordering rotates m/2 disjoint index pairs. Every CTA computes all of the round's
// rotations from the current A into its shared memory (they are cheap and identical
// everywhere), then applies its share of A' = J^T A J block by block (each 2 x 2 block (P, Q)
// depends only on its own four entries and the rotations of P and Q) into the other buffer of
// a double-buffered A, and V <- V J row by row in place: one grid barrier per round. The
// off-diagonal norm is reduced deterministically (per-CTA partials, summed in CTA order).
struct JacobiArgs {
  double* A;        // input matrix; on return the rotated matrix (diagonal = eigenvalues)
  double* A2;       // second buffer, m x m
  double* V;
  int m;
  int max_sweeps;
  double tol;
  double* partial;  // [2 * gridDim.x]
  int* done;        // [1]
};

__global__ void __launch_bounds__(256) jacobi_grid_kernel(JacobiArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double jsh[];
  const int m = a.m;
  const int mp = m + (m & 1);
  const int npairs = mp / 2;
  double* s_cs = jsh;
  double* s_sn = jsh + npairs;
  int* s_pp = reinterpret_cast<int*>(jsh + 2 * npairs);
  int* s_qq = s_pp + npairs;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  __shared__ double red[33];
  double* A = a.A;
  double* B = a.A2;
  for (long long idx = gtid; idx < (long long)m * m; idx += gstride)
    a.V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (long long idx = gtid; idx < (long long)m * m; idx += gstride) {
      const double v = A[idx];
      tot += v * v;
      if (idx / m != idx % m) off += v * v;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
      a.partial[2 * blockIdx.x] = off;
      a.partial[2 * blockIdx.x + 1] = tot;
    }
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double so = 0.0, st = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        so += a.partial[2 * b];
        st += a.partial[2 * b + 1];
      }
      a.done[0] = so <= a.tol * a.tol * st ? 1 : 0;
    }
    grid.sync();
    if (a.done[0]) break;
    for (int r = 0; r < mp - 1; ++r) {
      for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = 0;
          q = (r % (mp - 1)) + 1;
        } else {
          p = (i + r) % (mp - 1) + 1;
          q = (mp - 1 - i + r) % (mp - 1) + 1;
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sv = 0.0;
        if (q < m) {
          const double apq = A[(long long)p * m + q];
          if (apq != 0.0) {
            const double theta = (A[(long long)q * m + q] - A[(long long)p * m + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        s_pp[i] = p;
        s_qq[i] = q;
        s_cs[i] = c;
        s_sn[i] = sv;
      }
      __syncthreads();
      for (long long idx = gtid; idx < (long long)npairs * npairs; idx += gstride) {
        const int P = (int)(idx / npairs), Q = (int)(idx % npairs);
        const int p1 = s_pp[P], q1 = s_qq[P], p2 = s_pp[Q], q2 = s_qq[Q];
        const double c1 = s_cs[P], s1 = s_sn[P], c2 = s_cs[Q], s2 = s_sn[Q];
        const bool hq1 = q1 < m, hq2 = q2 < m;
        const double x00 = A[(long long)p1 * m + p2];
        const double x01 = hq2 ? A[(long long)p1 * m + q2] : 0.0;
        const double x10 = hq1 ? A[(long long)q1 * m + p2] : 0.0;
        const double x11 = (hq1 && hq2) ? A[(long long)q1 * m + q2] : 0.0;
        // rows (J^T A), then columns (A J)
        const double r00 = c1 * x00 - s1 * x10, r01 = c1 * x01 - s1 * x11;
        const double r10 = s1 * x00 + c1 * x10, r11 = s1 * x01 + c1 * x11;
        B[(long long)p1 * m + p2] = c2 * r00 - s2 * r01;
        if (hq2) B[(long long)p1 * m + q2] = s2 * r00 + c2 * r01;
        if (hq1) B[(long long)q1 * m + p2] = c2 * r10 - s2 * r11;
        if (hq1 && hq2) B[(long long)q1 * m + q2] = s2 * r10 + c2 * r11;
      }
      for (long long idx = gtid; idx < (long long)m * npairs; idx += gstride) {
        const int row = (int)(idx / npairs), Q = (int)(idx % npairs);
        const int p2 = s_pp[Q], q2 = s_qq[Q];
        if (q2 >= m) continue;
        const double c2 = s_cs[Q], s2 = s_sn[Q];
        const double vp = a.V[(long long)row * m + p2], vq = a.V[(long long)row * m + q2];
        a.V[(long long)row * m + p2] = c2 * vp - s2 * vq;
        a.V[(long long)row * m + q2] = s2 * vp + c2 * vq;
      }
      grid.sync();
      double* t = A;
      A = B;
      B = t;
    }
  }
  if (A != a.A) {   // an odd number of rounds ended in the second buffer
    for (long long idx = gtid; idx < (long long)m * m; idx += gstride) a.A[idx] = A[idx];
  }
}

// Sort eigenpairs ascending (stable in index), sign convention: the largest-|.| entry of each
// eigenvector (first on ties) is positive. evals[i] = A[i][i]; Vout columns sorted.
__global__ void sort_eig_kernel(const double* A, const double* V, int m, double* evals,
                                double* Vout) {
  extern __shared__ int rank[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ei = A[i * m + i];
    int r = 0;
    for (int j = 0; j < m; ++j) {
      const double ej = A[j * m + j];
      if (ej < ei || (ej == ei && j < i)) ++r;
    }
    rank[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int r = rank[i];
    evals[r] = A[i * m + i];
    int arg = 0;
    double best = -1.0;
    for (int j = 0; j < m; ++j)
      if (fabs(V[j * m + i]) > best) {
        best = fabs(V[j * m + i]);
        arg = j;
      }
    const double sg = V[arg * m + i] < 0.0 ? -1.0 : 1.0;
    for (int j = 0; j < m; ++j) Vout[j * m + r] = sg * V[j * m + i];
  }
}

// C (m1 x n1) = op(A)^T-free small dense products in float64: C[i][j] = sum_k A[i*sa + k*ka] *
// B[k*sb + j*jb]
__global__ void small_gemm_kernel(const double* A, long long a_i, long long a_k, const double* B,
                                  long long b_k, long long b_j, double* C, int m1, int n1, int K) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m1 * n1;
       idx += gridDim.x * blockDim.x) {
    const int i = idx / n1, j = idx % n1;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += A[i * a_i + k * a_k] * B[k * b_k + j * b_j];
    C[idx] = acc;
  }
}

// X[:, c] = U[:, keep[c]] / sqrt(mu[keep[c]])
__global__ void canon_basis_kernel(const double* U, const double* mu, const int* keep, int m,
                                   int k, double* X) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * k;
       idx += gridDim.x * blockDim.x) {
    const int i = idx / k, c = idx % k;
    X[idx] = U[i * m + keep[c]] / sqrt(mu[keep[c]]);
  }
}

// Sign convention of the Ritz vectors: the largest-|.| entry of each column (first on ties) is
// made positive. V is m x n row-major; one thread per column.
__global__ void fix_sign_kernel(double* V, int m, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int arg = 0;
  double best = -1.0;
  for (int i = 0; i < m; ++i)
    if (fabs(V[(long long)i * n + j]) > best) {
      best = fabs(V[(long long)i * n + j]);
      arg = i;
    }
  if (V[(long long)arg * n + j] < 0.0)
    for (int i = 0; i < m; ++i) V[(long long)i * n + j] = -V[(long long)i * n + j];
}

__global__ void symmetrize_kernel(double* A, int m) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += gridDim.x * blockDim.x) {
    const int i = idx / m, j = idx % m;
    if (i < j) {
      const double v = 0.5 * (A[i * m + j] + A[j * m + i]);
      A[i * m + j] = v;
      A[j * m + i] = v;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// host-side drivers
// ------------------------------------------------------------------------------------------------
// Scratch (in doubles) of one grid Jacobi solve of size m: rotations, pairs, partial sums.
static size_t jacobi_scratch_doubles(int m) { return (size_t)m * m + 2 * 1024 + 8; }

// Shared memory of jacobi_grid_kernel: the round's rotations (cos, sin, p, q per pair).
static size_t jacobi_smem(int m) {
  const int npairs = (m + (m & 1)) / 2;
  return (size_t)npairs * (2 * sizeof(double) + 2 * sizeof(int));
}
constexpr int kJacobiMaxM = 2048;

static int jacobi_grid_blocks(int device) {
  static int cached[64] = {0};
  if (device >= 0 && device < 64 && cached[device]) return cached[device];
  int per_sm = 0, sms = 0;
  CUDA_CHECK(cudaFuncSetAttribute(jacobi_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)jacobi_smem(kJacobiMaxM)));
  CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel, 256,
                                                           jacobi_smem(kJacobiMaxM)));
  CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  // one CTA per SM: measured on the 300 x 300 Rayleigh-Ritz of block LOBPCG, two per SM made
  // each grid barrier dearer (55 ms against 42 ms per call) and half as many made each round's
  // share of the rotations dearer (55 ms)
  int b = std::max(1, std::min(per_sm, 1) * sms);
  b = std::min(b, 1024);
  if (device >= 0 && device < 64) cached[device] = b;
  return b;
}

// Eigen-decomposition of the symmetric m x m matrix A (destroyed: diagonal = eigenvalues) with
// eigenvectors in the columns of V, on the whole GPU. scratch: jacobi_scratch_doubles(m).
static void launch_jacobi_grid(ttn_ctx* ctx, double* A, double* V, int m, double* scratch) {
  TTN_REQUIRE(m <= kJacobiMaxM, "Jacobi eigensolver: m = %d above %d", m, kJacobiMaxM);
  JacobiArgs a;
  a.A = A;
  a.A2 = scratch;
  a.V = V;
  a.m = m;
  a.max_sweeps = 40;
  a.tol = 1e-15;
  a.partial = scratch + (size_t)m * m;
  a.done = reinterpret_cast<int*>(scratch + (size_t)m * m + 2 * 1024);
  const int blocks = jacobi_grid_blocks(ctx->device);
  void* args[] = {&a};
  CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)jacobi_grid_kernel, dim3(blocks), dim3(256),
                                         args, jacobi_smem(m), ctx->stream));
}


template <class T> T* work_node(ttn_block* b, int t);
template <> double* work_node<double>(ttn_block* b, int t) {
  b->touch();
  return b->node64(t);
}
template <> float* work_node<float>(ttn_block* b, int t) {
  b->node32(t);
  return b->d32.as<float>() + b->off[t];
}
template <class T> void commit(ttn_block* b);
template <> void commit<double>(ttn_block* b) { b->touch(); }
template <> void commit<float>(ttn_block* b) {
  b->node32(0);
  launch_to_f64(b->ctx, b->d32.as<float>(), b->d64.as<double>(), b->total);
  b->f32_valid = true;
}

struct DevVec {
  DevBuf buf;
  int maxv = 0;
  int n = 0;
  DevVec() = default;
  template <class V>
  DevVec(const std::vector<V>& v, cudaStream_t s)
      : buf(std::max<size_t>(v.size(), 1) * sizeof(V), s), n((int)v.size()) {
    if (!v.empty())
      CUDA_CHECK(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice,
                                 s));
  }
};

static PairSet make_pairs(const std::vector<int>& pb, const std::vector<int>& pk, DevVec& db,
                          DevVec& dk, cudaStream_t s) {
  db = DevVec(pb, s);
  dk = DevVec(pk, s);
  PairSet ps;
  ps.P = (int)pb.size();
  ps.d_pb = db.buf.as<int>();
  ps.d_pk = dk.buf.as<int>();
  for (int x : pb) ps.max_bra = std::max(ps.max_bra, x);
  for (int x : pk) ps.max_ket = std::max(ps.max_ket, x);
  return ps;
}

// Environments of <bra|H|ket> over a fixed pair list, computed on demand and invalidated when
// node tensors change (an up environment depends on the subtree below its edge, a down
// environment on everything outside it).
template <class T>
struct EnvCache {
  ttn_ctx* ctx = nullptr;
  ttn_ttno* H = nullptr;
  const ttn_block* bra = nullptr;
  const ttn_block* ket = nullptr;
  PairSet ps;
  DevVec dpb, dpk;
  const TreeInfo* tr = nullptr;
  std::vector<DevBuf> up, down;
  std::vector<char> up_ok, down_ok;
  std::vector<std::vector<char>> in_sub;

  void init(ttn_ctx* c, ttn_ttno* h, const ttn_block* b, const ttn_block* k,
            const std::vector<int>& pb, const std::vector<int>& pk) {
    ctx = c;
    H = h;
    bra = b;
    ket = k;
    tr = &b->tree;
    ps = make_pairs(pb, pk, dpb, dpk, c->stream);
    up.clear();
    down.clear();
    up.resize(tr->n);
    down.resize(tr->n);
    up_ok.assign(tr->n, 0);
    down_ok.assign(tr->n, 0);
    in_sub.assign(tr->n, std::vector<char>(tr->n, 0));
    for (int e = 0; e < tr->n; ++e) {
      std::vector<int> st{e};
      while (!st.empty()) {
        int u = st.back();
        st.pop_back();
        in_sub[e][u] = 1;
        for (int ch : tr->children[u]) st.push_back(ch);
      }
    }
  }
  long long esize(int e) const { return (long long)H->wbond[e] * bra->bond[e] * ket->bond[e]; }
  void invalidate(int u) {
    for (int e = 0; e < tr->n; ++e) {
      if (e == tr->root) continue;
      if (in_sub[e][u]) up_ok[e] = 0;
      else down_ok[e] = 0;
    }
  }
  const T* get_up(int e) {
    if (!up_ok[e]) {
      const int nl = tr->nlegs(e);
      std::vector<const T*> env(nl, nullptr);
      for (int m = 1; m < nl; ++m) env[m] = get_up(tr->legs[e][m]);
      const long long n = (long long)ps.P * esize(e);
      if (!up[e].p) up[e] = DevBuf((size_t)n * sizeof(T), ctx->stream);
      node_op<T>(ctx, H, e, 0, bra, ket, ps, env, {}, up[e].p, n, OUT_ENV);
      up_ok[e] = 1;
    }
    return up[e].as<T>();
  }
  const T* get_down(int e) {
    if (!down_ok[e]) {
      const int u = tr->parent[e];
      const int nl = tr->nlegs(u);
      const int m = tr->leg_to(u, e);
      std::vector<const T*> env(nl, nullptr);
      const int off = u == tr->root ? 0 : 1;
      if (off) env[0] = get_down(u);
      for (int m2 = off; m2 < nl; ++m2)
        if (m2 != m) env[m2] = get_up(tr->legs[u][m2]);
      const long long n = (long long)ps.P * esize(e);
      if (!down[e].p) down[e] = DevBuf((size_t)n * sizeof(T), ctx->stream);
      node_op<T>(ctx, H, u, m, bra, ket, ps, env, {}, down[e].p, n, OUT_ENV);
      down_ok[e] = 1;
    }
    return down[e].as<T>();
  }
  std::vector<const T*> node_envs(int t) {
    const int nl = tr->nlegs(t);
    std::vector<const T*> env(nl);
    for (int m = 0; m < nl; ++m) {
      const int nb = tr->legs[t][m];
      env[m] = tr->parent[t] == nb ? get_down(t) : get_up(nb);
    }
    return env;
  }
};

// Move the orthogonality centre of every state of `b` from node u to its neighbour v.
template <class T>
static void qr_move(ttn_ctx* ctx, ttn_block* b, int u, int v) {
  const TreeInfo& tr = b->tree;
  cudaStream_t st = ctx->stream;
  const int n = b->n_states;
  if (n == 0) return;
  const int nl = tr.nlegs(u);
  const int m = tr.leg_to(u, v);
  const int D = b->bdim(u, m);
  const long long size = b->size[u];
  const long long rows = size / D;
  TTN_REQUIRE(rows >= D, "gauge move %d->%d: bond %d exceeds the rest of the node (%lld)", u, v,
              D, rows);
  TTN_REQUIRE(D <= 64, "gauge move: bonds above 64 are not supported (%d)", D);
  std::vector<int> dims(b->dims[u].begin(), b->dims[u].end());   // legs..., phys
  std::vector<int> perm;
  for (int k = 0; k <= nl; ++k)
    if (k != m) perm.push_back(k);
  perm.push_back(m);
  T* node = work_node<T>(b, u);
  DevBuf M((size_t)n * size * sizeof(T), st), Q((size_t)n * size * sizeof(T), st),
      R((size_t)n * D * D * sizeof(T), st);
  launch_permute<T>(ctx, node, M.as<T>(), n, nl + 1, dims.data(), perm.data());
  {
    LaunchScope ls(ctx, sizeof(T) == 8 ? "householder_qr_f64" : "householder_qr_f32",
                   4.0 * rows * D * D * n, 4.0 * sizeof(T) * size * n);
    // working copies on chip when both fit (c2 backbone: 576 x 24 float32 = 55 KB each)
    const size_t smem = 2 * (size_t)rows * D * sizeof(T);
    const bool on_chip = smem <= 200 * 1024;
    if (on_chip)
      CUDA_CHECK(cudaFuncSetAttribute(householder_qr_kernel<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    householder_qr_kernel<T><<<n, kT, on_chip ? smem : 0, st>>>(
        M.as<T>(), Q.as<T>(), R.as<T>(), (int)rows, D, size, on_chip ? 1 : 0);
    CUDA_LAUNCH_CHECK();
  }
  std::vector<int> pdims(nl + 1), inv(nl + 1);
  for (int k = 0; k <= nl; ++k) {
    pdims[k] = dims[perm[k]];
    inv[perm[k]] = k;
  }
  launch_permute<T>(ctx, Q.as<T>(), node, n, nl + 1, pdims.data(), inv.data());
  // absorb R into v's leg toward u
  const int mv = tr.leg_to(v, u);
  long long inner = 1;
  for (size_t k = mv + 1; k < b->dims[v].size(); ++k) inner *= b->dims[v][k];
  const long long vsize = b->size[v];
  T* vnode = work_node<T>(b, v);
  DevBuf tmp((size_t)n * vsize * sizeof(T), st);
  {
    LaunchScope ls(ctx, "leg_product", 2.0 * D * vsize * n, 2.0 * sizeof(T) * vsize * n);
    leg_product_kernel<T><<<grid_of((long long)n * vsize), kT, 0, st>>>(
        R.as<T>(), vnode, tmp.as<T>(), n, vsize, inner, D);
    CUDA_LAUNCH_CHECK();
  }
  CUDA_CHECK(cudaMemcpyAsync(vnode, tmp.p, (size_t)n * vsize * sizeof(T),
                             cudaMemcpyDeviceToDevice, st));
}

template <class T>
static void canonicalize(ttn_ctx* ctx, ttn_block* b) {
  for (int c : b->tree.post)
    if (c != b->tree.root) qr_move<T>(ctx, b, c, b->tree.parent[c]);
}

template <class T, class F>
static int move_center(ttn_ctx* ctx, ttn_block* b, int from, int to, F&& on_change) {
  std::vector<int> p = b->tree.path(from, to);
  for (size_t k = 0; k + 1 < p.size(); ++k) {
    qr_move<T>(ctx, b, p[k], p[k + 1]);
    on_change(p[k]);
    on_change(p[k + 1]);
  }
  return to;
}

template <class T>
static void launch_dot(ttn_ctx* ctx, const T* x, const T* y, long long n, int n_states,
                       double* out) {
  if (n_states == 0) return;
  LaunchScope ls(ctx, "dot", 2.0 * n * n_states, 2.0 * sizeof(T) * n * n_states);
  dot_kernel<T><<<n_states, kT, 0, ctx->stream>>>(x, y, n, out);
  CUDA_LAUNCH_CHECK();
}

template <class T>
static void launch_scale(ttn_ctx* ctx, T* x, const double* f, long long n, int mode,
                         int n_states) {
  if (n_states == 0) return;
  LaunchScope ls(ctx, "scale", 1.0 * n * n_states, 2.0 * sizeof(T) * n * n_states);
  scale_kernel<T><<<grid_of(n * n_states), kT, 0, ctx->stream>>>(x, f, n, mode, n_states);
  CUDA_LAUNCH_CHECK();
}

// Batched MINRES on (H_eff,t - shift_s) x_s = b_s for all states s; x holds the warm start.
// Returns true if some state hit maxiter without reaching the tolerance.
template <class T>
static bool minres_batched(ttn_ctx* ctx, ttn_ttno* H, EnvCache<T>& env, int t,
                           const ttn_block* shape, T* x, const T* b, const double* d_shift,
                           int n, int maxiter, double tol) {
  cudaStream_t st = ctx->stream;
  const long long sz = shape->size[t];
  const long long total = sz * n;
  std::vector<DevBuf> bufs;
  for (int i = 0; i < 5; ++i) bufs.emplace_back((size_t)std::max<long long>(total, 1) * sizeof(T), st);
  T* p = bufs[0].as<T>();
  T* v = bufs[1].as<T>();
  T* vp = bufs[2].as<T>();
  T* w1 = bufs[3].as<T>();
  T* w2 = bufs[4].as<T>();
  DevBuf sc((size_t)n * MR_NFIELDS * sizeof(double), st), d1(n * sizeof(double), st),
      d2(n * sizeof(double), st), d3(n * sizeof(double), st);
  const double eps_t = sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
  std::vector<const T*> envs = env.node_envs(t);
  std::vector<int> da(shape->tree.nlegs(t));
  for (int m = 0; m < (int)da.size(); ++m) da[m] = shape->bdim(t, m);
  auto matvec = [&](const T* in, T* out) {
    node_op<T>(ctx, H, t, -1, nullptr, shape, env.ps, envs, da, out, total, OUT_LOCAL, in, n);
    launch_shift_axpy<T>(ctx, out, in, d_shift, n, sz);
  };
  matvec(x, p);
  {
    LaunchScope ls(ctx, "minres_vec", 1.0 * total, 3.0 * sizeof(T) * total);
    sub_kernel<T><<<grid_of(total), kT, 0, st>>>(b, p, total);
    CUDA_LAUNCH_CHECK();
  }
  launch_dot<T>(ctx, b, b, sz, n, d1.as<double>());
  launch_dot<T>(ctx, p, p, sz, n, d2.as<double>());
  {
    LaunchScope ls(ctx, "minres_scalar", 0.0, 0.0);
    mr_init_scalars<<<(n + 127) / 128, 128, 0, st>>>(sc.as<double>(), d1.as<double>(),
                                                     d2.as<double>(), n);
    CUDA_LAUNCH_CHECK();
  }
  {
    // p holds r = b - A x0; rebuild the recurrence vectors from it (b - (b - r) = r)
    LaunchScope ls(ctx, "minres_vec", 1.0 * total, 6.0 * sizeof(T) * total);
    DevBuf zero((size_t)std::max<long long>(total, 1) * sizeof(T), st);
    CUDA_CHECK(cudaMemsetAsync(zero.p, 0, total * sizeof(T), st));
    mr_init_vectors<T><<<grid_of(total), kT, 0, st>>>(sc.as<double>(), p, zero.as<T>(), v, vp,
                                                      w1, w2, sz, n);
    CUDA_LAUNCH_CHECK();
  }
  // One MINRES step touches only device state at fixed addresses, so it is captured once as a
  // CUDA graph and replayed (the planning work of the contraction runs once, at capture).
  auto one_step = [&]() {
    matvec(v, p);
    launch_dot<T>(ctx, v, p, sz, n, d1.as<double>());
    {
      LaunchScope ls(ctx, "minres_vec", 4.0 * total, 4.0 * sizeof(T) * total);
      mr_lanczos<T><<<grid_of(total), kT, 0, st>>>(sc.as<double>(), d1.as<double>(), p, v, vp,
                                                   sz, n);
      CUDA_LAUNCH_CHECK();
    }
    launch_dot<T>(ctx, p, p, sz, n, d2.as<double>());
    {
      LaunchScope ls(ctx, "minres_scalar", 0.0, 0.0);
      mr_step_scalars<<<(n + 127) / 128, 128, 0, st>>>(sc.as<double>(), d1.as<double>(),
                                                       d2.as<double>(), n, tol, maxiter);
      CUDA_LAUNCH_CHECK();
    }
    {
      LaunchScope ls(ctx, "minres_vec", 8.0 * total, 8.0 * sizeof(T) * total);
      mr_step_vectors<T><<<grid_of(total), kT, 0, st>>>(sc.as<double>(), x, v, vp, w1, w2, p,
                                                        sz, n);
      CUDA_LAUNCH_CHECK();
    }
    launch_dot<T>(ctx, x, x, sz, n, d3.as<double>());
    {
      LaunchScope ls(ctx, "minres_scalar", 0.0, 0.0);
      mr_floor_check<<<(n + 127) / 128, 128, 0, st>>>(sc.as<double>(), d3.as<double>(), n, eps_t);
      CUDA_LAUNCH_CHECK();
    }
  };
  cudaGraphExec_t exec = nullptr;
  long long step_launches = 0;
  double step_flops = 0.0;
  if (maxiter > 1) {
    cudaGraph_t graph = nullptr;
    const long long l0 = ctx->launches;
    const double f0 = ctx->flops_total;
    CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    try {
      one_step();
    } catch (...) {
      ctx->capturing = false;
      cudaStreamEndCapture(st, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    ctx->capturing = false;
    CUDA_CHECK(cudaStreamEndCapture(st, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_CHECK(ie);
    step_launches = ctx->launches - l0;
    step_flops = ctx->flops_total - f0;
    ctx->launches = l0;
    ctx->flops_total = f0;
  }
  struct ExecGuard {
    cudaGraphExec_t e;
    ~ExecGuard() {
      if (e) cudaGraphExecDestroy(e);
    }
  } exec_guard{exec};
  for (int it = 0; it < maxiter; ++it) {
    if (exec) {
      CUDA_CHECK(cudaGraphLaunch(exec, st));
      ctx->launches += step_launches;
      ctx->flops_total += step_flops;
    } else {
      one_step();
    }
    if (maxiter > 32 && (it + 1) % 16 == 0) {
      std::vector<double> h((size_t)n * MR_NFIELDS);
      CUDA_CHECK(cudaMemcpyAsync(h.data(), sc.p, h.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
      CUDA_CHECK(cudaStreamSynchronize(st));
      bool any = false;
      for (int s = 0; s < n; ++s) any |= h[(size_t)s * MR_NFIELDS + MR_ACTIVE] != 0.0;
      if (!any) break;
    }
  }
  std::vector<double> h((size_t)n * MR_NFIELDS);
  CUDA_CHECK(cudaMemcpyAsync(h.data(), sc.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  bool hit = false;
  for (int s = 0; s < n; ++s) {
    const double* f = h.data() + (size_t)s * MR_NFIELDS;
    hit |= f[MR_ACTIVE] != 0.0 || f[MR_HITCAP] != 0.0;
  }
  return hit;
}

// ALS (Sec. II.C.3): y_s <- argmin over one node at a time of |(H - shift_s) y_s - rhs_s|.
template <class T>
static bool als_impl(ttn_ctx* ctx, ttn_ttno* H, const std::vector<double>& shift,
                     const ttn_block* rhs, ttn_block* y, int n_sweeps, int mr_max,
                     double mr_tol) {
  const TreeInfo& tr = y->tree;
  const int n = y->n_states;
  cudaStream_t st = ctx->stream;
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  canonicalize<T>(ctx, y);
  int center = tr.root;
  EnvCache<T> eH, eS;
  eH.init(ctx, H, y, y, id, id);
  eS.init(ctx, identity_for(ctx, tr), y, rhs, id, id);
  DevVec dshift(shift, st);
  bool hit = false;
  for (int sweep = 0; sweep < n_sweeps; ++sweep) {
    for (int t : tr.pre) {
      center = move_center<T>(ctx, y, center, t, [&](int u) {
        eH.invalidate(u);
        eS.invalidate(u);
      });
      const long long sz = y->size[t];
      DevBuf bvec((size_t)std::max<long long>(sz * n, 1) * sizeof(T), st);
      std::vector<int> da(tr.nlegs(t));
      for (int m = 0; m < (int)da.size(); ++m) da[m] = y->bdim(t, m);
      node_op<T>(ctx, eS.H, t, -1, nullptr, rhs, eS.ps, eS.node_envs(t), da, bvec.p, sz * n,
                 OUT_LOCAL);
      T* x = work_node<T>(y, t);
      hit |= minres_batched<T>(ctx, H, eH, t, y, x, bvec.as<T>(), dshift.buf.as<double>(), n,
                               mr_max, mr_tol);
      eH.invalidate(t);
      eS.invalidate(t);
    }
  }
  commit<T>(y);
  CUDA_CHECK(cudaStreamSynchronize(st));
  return hit;
}

struct FitGroup {
  ttn_ttno* op;
  const ttn_block* in;
  std::vector<int> out_j, in_k;   // pairs, sorted by out_j
  std::vector<double> coef;
};

// Variational fitting (Sec. II.C.2): in canonical gauge the local solution at the centre is
// the right-hand side sum_i c_i <psi without t| O_i |phi_i>.
template <class T>
static void fit_impl(ttn_ctx* ctx, std::vector<FitGroup>& groups, ttn_block* out, int n_sweeps) {
  const TreeInfo& tr = out->tree;
  const int n_out = out->n_states;
  cudaStream_t st = ctx->stream;
  canonicalize<T>(ctx, out);
  int center = tr.root;
  std::vector<EnvCache<T>> caches(groups.size());
  std::vector<DevVec> seg(groups.size()), coef(groups.size());
  for (size_t g = 0; g < groups.size(); ++g) {
    caches[g].init(ctx, groups[g].op, out, groups[g].in, groups[g].out_j, groups[g].in_k);
    std::vector<int> sp(n_out + 1, 0);
    for (int j : groups[g].out_j) sp[j + 1]++;
    for (int j = 0; j < n_out; ++j) sp[j + 1] += sp[j];
    seg[g] = DevVec(sp, st);
    coef[g] = DevVec(groups[g].coef, st);
  }
  for (int sweep = 0; sweep < n_sweeps; ++sweep) {
    for (int t : tr.pre) {
      center = move_center<T>(ctx, out, center, t, [&](int u) {
        for (auto& c : caches) c.invalidate(u);
      });
      const long long sz = out->size[t];
      DevBuf acc((size_t)std::max<long long>(sz * n_out, 1) * sizeof(T), st);
      CUDA_CHECK(cudaMemsetAsync(acc.p, 0, (size_t)sz * n_out * sizeof(T), st));
      std::vector<int> da(tr.nlegs(t));
      for (int m = 0; m < (int)da.size(); ++m) da[m] = out->bdim(t, m);
      for (size_t g = 0; g < groups.size(); ++g) {
        const int P = caches[g].ps.P;
        if (P == 0) continue;
        DevBuf Y((size_t)P * sz * sizeof(T), st);
        node_op<T>(ctx, groups[g].op, t, -1, nullptr, groups[g].in, caches[g].ps,
                   caches[g].node_envs(t), da, Y.p, (long long)P * sz, OUT_LOCAL);
        LaunchScope ls(ctx, "seg_sum", 2.0 * P * sz, sizeof(T) * ((double)P * sz + 2.0 * n_out * sz));
        seg_sum_kernel<T><<<grid_of(sz * n_out), kT, 0, st>>>(
            Y.as<T>(), seg[g].buf.as<int>(), coef[g].buf.as<double>(), acc.as<T>(), n_out, sz, 1);
        CUDA_LAUNCH_CHECK();
      }
      T* node = work_node<T>(out, t);
      CUDA_CHECK(cudaMemcpyAsync(node, acc.p, (size_t)sz * n_out * sizeof(T),
                                 cudaMemcpyDeviceToDevice, st));
      for (auto& c : caches) c.invalidate(t);
    }
  }
  commit<T>(out);
  CUDA_CHECK(cudaStreamSynchronize(st));
}

// Scale every state to unit norm (the norm is taken over the whole network).
template <class T>
static void normalize_states(ttn_ctx* ctx, ttn_block* b, int prec) {
  const int n = b->n_states;
  DevBuf S((size_t)n * sizeof(double), ctx->stream);
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  gram_pairs<T>(ctx, identity_for(ctx, b->tree), b, b, id, id, S.as<double>());
  (void)prec;
  launch_scale<double>(ctx, b->node64(b->tree.root), S.as<double>(), b->size[b->tree.root], 1, n);
  b->touch();
  CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
}

// Rayleigh-Ritz on device data (float64): theta[n], V[m x n] (device).
static void rayleigh_ritz_device(ttn_ctx* ctx, int m, const double* dHt, const double* dMt,
                                 int n, double eps, double* d_theta, double* dV) {
  cudaStream_t st = ctx->stream;
  TTN_REQUIRE(m >= 1 && n >= 1 && n <= m, "rayleigh_ritz: need 1 <= n <= m");
  TTN_REQUIRE(m <= 2048, "rayleigh_ritz: m = %d too large", m);
  const size_t mm = (size_t)m * m;
  DevBuf A(mm * sizeof(double), st), U(mm * sizeof(double), st), Us(mm * sizeof(double), st),
      mu(m * sizeof(double), st);
  DevBuf jac(jacobi_scratch_doubles(m) * sizeof(double), st);
  auto eig = [&](double* Ain, int k, double* evals, double* Vout) {
    {
      LaunchScope ls(ctx, "symmetrize", 0.0, 16.0 * k * k);
      symmetrize_kernel<<<grid_of((long long)k * k), kT, 0, st>>>(Ain, k);
      CUDA_LAUNCH_CHECK();
    }
    {
      LaunchScope ls(ctx, "jacobi_grid_f64", 0.0, 0.0);
      launch_jacobi_grid(ctx, Ain, U.as<double>(), k, jac.as<double>());
    }
    {
      LaunchScope ls(ctx, "sort_eig", 0.0, 0.0);
      sort_eig_kernel<<<1, 256, k * sizeof(int), st>>>(Ain, U.as<double>(), k, evals, Vout);
      CUDA_LAUNCH_CHECK();
    }
  };
  CUDA_CHECK(cudaMemcpyAsync(A.p, dMt, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
  eig(A.as<double>(), m, mu.as<double>(), Us.as<double>());
  std::vector<double> hmu(m);
  CUDA_CHECK(cudaMemcpyAsync(hmu.data(), mu.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  for (double x : hmu)
    if (!std::isfinite(x)) TTN_FAIL(TTN_ENONFINITE, "rayleigh_ritz: non-finite overlap matrix");
  const double mx = *std::max_element(hmu.begin(), hmu.end());
  std::vector<int> keep;
  for (int i = 0; i < m; ++i)
    if (hmu[i] > eps * mx) keep.push_back(i);
  const int k = (int)keep.size();
  TTN_REQUIRE(k >= n, "rayleigh_ritz: only %d of %d directions survive eps = %g", k, n, eps);
  DevVec dkeep(keep, st);
  DevBuf X((size_t)m * k * sizeof(double), st), HX((size_t)m * k * sizeof(double), st),
      Hp((size_t)k * k * sizeof(double), st), th(k * sizeof(double), st),
      Y((size_t)k * k * sizeof(double), st);
  {
    LaunchScope ls(ctx, "rr_small", 0.0, 0.0);
    canon_basis_kernel<<<grid_of((long long)m * k), kT, 0, st>>>(Us.as<double>(), mu.as<double>(),
                                                               dkeep.buf.as<int>(), m, k,
                                                               X.as<double>());
    CUDA_LAUNCH_CHECK();
    // HX = Ht X   (m x k)
    small_gemm_kernel<<<grid_of((long long)m * k), kT, 0, st>>>(dHt, m, 1, X.as<double>(), k, 1,
                                                              HX.as<double>(), m, k, m);
    // Hp = X^T HX (k x k)
    small_gemm_kernel<<<grid_of((long long)k * k), kT, 0, st>>>(X.as<double>(), 1, k,
                                                              HX.as<double>(), k, 1,
                                                              Hp.as<double>(), k, k, m);
    CUDA_LAUNCH_CHECK();
  }
  eig(Hp.as<double>(), k, th.as<double>(), Y.as<double>());
  {
    LaunchScope ls(ctx, "rr_small", 0.0, 0.0);
    // V = X Y[:, :n]   (m x n)
    small_gemm_kernel<<<grid_of((long long)m * n), kT, 0, st>>>(X.as<double>(), k, 1,
                                                              Y.as<double>(), k, 1, dV, m, n, k);
    fix_sign_kernel<<<(n + 127) / 128, 128, 0, st>>>(dV, m, n);
    CUDA_LAUNCH_CHECK();
  }
  CUDA_CHECK(cudaMemcpyAsync(d_theta, th.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
}

template <class F>
static ttn_status guarded_s(ttn_ctx* ctx, F&& f) {
  try {
    ttn_status s = f();
    if (s == TTN_OK) ctx->last_error.clear();
    return s;
  } catch (const TtnError& e) {
    ctx->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->last_error = "host allocation failed";
    return TTN_ENOMEM;
  }
}

static void check_block_like(const ttn_block* a, const ttn_block* b) {
  TTN_REQUIRE(a && b, "NULL block");
  TTN_REQUIRE(a->tree.same_shape(b->tree) && a->bond == b->bond,
              "blocks differ in tree or bond dimensions");
}

template <class T>
static void lobpcg_impl(ttn_ctx* ctx, ttn_ttno* H, ttn_block* x, int n_iter, double shift_offset,
                        int als_sweeps, int mr_max, double mr_tol, int fit_sweeps, int prec,
                        double* eig_hist, bool& hit) {
  const TreeInfo& tr = x->tree;
  const int n = x->n_states;
  cudaStream_t st = ctx->stream;
  ttn_ttno* Id = identity_for(ctx, tr);
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  auto new_block = [&](int ns) {
    ttn_tree tmp;
    tmp.ctx = ctx;
    tmp.info = tr;
    ttn_block* b = nullptr;
    ttn_status s = ttn_block_create(ctx, &tmp, ns, x->bond.data(), &b);
    if (s != TTN_OK) TTN_FAIL(s, "%s", ctx->last_error.c_str());
    return std::unique_ptr<ttn_block>(b);
  };
  iter_clock_start(ctx);
  normalize_states<T>(ctx, x, prec);
  std::vector<double> lam(n);
  {
    DevBuf hv((size_t)n * sizeof(double), st), sv((size_t)n * sizeof(double), st);
    gram_pairs<T>(ctx, H, x, x, id, id, hv.as<double>());
    gram_pairs<T>(ctx, Id, x, x, id, id, sv.as<double>());
    std::vector<double> h(n), s(n);
    CUDA_CHECK(cudaMemcpyAsync(h.data(), hv.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(s.data(), sv.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) lam[j] = h[j] / s[j];
  }
  if (eig_hist) std::copy(lam.begin(), lam.end(), eig_hist);
  iter_clock_mark(ctx);
  auto R = new_block(n), Y = new_block(n), P = new_block(n), Xn = new_block(n), Pn = new_block(n);
  bool have_p = false;
  const double rr_eps = prec == TTN_FP64 ? 1e-12 : 1e-6;
  for (int it = 1; it <= n_iter; ++it) {
    const double s = *std::min_element(lam.begin(), lam.end()) + shift_offset;
    // residual r_j = H x_j - lambda_j x_j by fitting, starting from x_j
    {
      PhaseScope ph(ctx, "residual_fit");
      std::vector<int> ids(n);
      std::iota(ids.begin(), ids.end(), 0);
      CUDA_CHECK(cudaStreamSynchronize(st));
      ttn_status cs = ttn_block_copy_states(R.get(), x, n, ids.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      std::vector<FitGroup> g(2);
      g[0] = {H, x, id, id, std::vector<double>(n, 1.0)};
      std::vector<double> ml(n);
      for (int j = 0; j < n; ++j) ml[j] = -lam[j];
      g[1] = {Id, x, id, id, ml};
      fit_impl<T>(ctx, g, R.get(), fit_sweeps);
    }
    // preconditioner: (H - s) y = r by ALS, starting from r
    {
      PhaseScope ph(ctx, "als_precondition");
      std::vector<int> ids(n);
      std::iota(ids.begin(), ids.end(), 0);
      ttn_status cs = ttn_block_copy_states(Y.get(), R.get(), n, ids.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      hit |= als_impl<T>(ctx, H, std::vector<double>(n, s), R.get(), Y.get(), als_sweeps, mr_max,
                         mr_tol);
    }
    // subspace S = {x} u {r} (u {p})
    const int m = have_p ? 3 * n : 2 * n;
    auto S = new_block(m);
    {
      // S = x, y, p in that order: each node's three slabs are contiguous copies
      for (int t = 0; t < tr.n; ++t) {
        const size_t bytes = (size_t)n * x->size[t] * sizeof(double);
        double* dst = S->node64(t);
        CUDA_CHECK(cudaMemcpyAsync(dst, x->node64(t), bytes, cudaMemcpyDeviceToDevice, st));
        CUDA_CHECK(cudaMemcpyAsync(dst + (long long)n * x->size[t], Y->node64(t), bytes,
                                   cudaMemcpyDeviceToDevice, st));
        if (have_p)
          CUDA_CHECK(cudaMemcpyAsync(dst + 2LL * n * x->size[t], P->node64(t), bytes,
                                     cudaMemcpyDeviceToDevice, st));
      }
      S->touch();
    }
    DevBuf Ht((size_t)m * m * sizeof(double), st), Mt((size_t)m * m * sizeof(double), st);
    CUDA_CHECK(cudaMemsetAsync(Ht.p, 0, (size_t)m * m * sizeof(double), st));
    CUDA_CHECK(cudaMemsetAsync(Mt.p, 0, (size_t)m * m * sizeof(double), st));
    {
      PhaseScope ph(ctx, "gram_H");
      if (gram_device(ctx, H, S.get(), S.get(), Ht.as<double>(), m, prec))
        TTN_FAIL(TTN_ENONFINITE, "LOBPCG iteration %d: non-finite <s_k|H|s_l>", it);
    }
    {
      PhaseScope ph(ctx, "gram_S");
      if (gram_device(ctx, Id, S.get(), S.get(), Mt.as<double>(), m, prec))
        TTN_FAIL(TTN_ENONFINITE, "LOBPCG iteration %d: non-finite <s_k|s_l>", it);
    }
    DevBuf th((size_t)n * sizeof(double), st), V((size_t)m * n * sizeof(double), st);
    {
      PhaseScope ph(ctx, "rayleigh_ritz");
      rayleigh_ritz_device(ctx, m, Ht.as<double>(), Mt.as<double>(), n, rr_eps, th.as<double>(),
                           V.as<double>());
    }
    std::vector<double> hth(n), hV((size_t)m * n);
    CUDA_CHECK(cudaMemcpyAsync(hth.data(), th.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(hV.data(), V.p, hV.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    // x_j = sum_k v_kj s_k (normalised), p_j = sum_{k >= n} v_kj s_k
    // x_j and p_j are fitted in one batch of 2n output states (outputs 0..n-1: x_j from all of
    // S; outputs n..2n-1: p_j from the states k >= n); every output's fit is independent.
    {
      PhaseScope ph(ctx, "fit_xp");
      auto XP = new_block(2 * n);
      std::vector<int> init(2 * n);
      FitGroup g{Id, S.get(), {}, {}, {}};
      for (int half = 0; half < 2; ++half) {
        const int k0 = half * n;
        for (int j = 0; j < n; ++j) {
          int arg = k0;
          double best = -1.0;
          for (int k = k0; k < m; ++k) {
            const double c = hV[(size_t)k * n + j];
            if (std::fabs(c) > best) {
              best = std::fabs(c);
              arg = k;
            }
            if (c != 0.0) {
              g.out_j.push_back(half * n + j);
              g.in_k.push_back(k);
              g.coef.push_back(c);
            }
          }
          init[half * n + j] = arg;
        }
      }
      ttn_status cs = ttn_block_copy_states(XP.get(), S.get(), 2 * n, init.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      std::vector<FitGroup> gs{g};
      fit_impl<T>(ctx, gs, XP.get(), fit_sweeps);
      std::vector<int> lo(n), hi(n);
      std::iota(lo.begin(), lo.end(), 0);
      std::iota(hi.begin(), hi.end(), n);
      cs = ttn_block_copy_states(Xn.get(), XP.get(), n, lo.data());
      if (cs == TTN_OK) cs = ttn_block_copy_states(Pn.get(), XP.get(), n, hi.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      normalize_states<T>(ctx, Xn.get(), prec);
    }
    std::swap(P, Pn);
    have_p = true;
    {
      std::vector<int> ids(n);
      std::iota(ids.begin(), ids.end(), 0);
      ttn_status cs = ttn_block_copy_states(x, Xn.get(), n, ids.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
    }
    lam = hth;
    if (eig_hist) std::copy(lam.begin(), lam.end(), eig_hist + (size_t)it * n);
    iter_clock_mark(ctx);
  }
  CUDA_CHECK(cudaStreamSynchronize(st));
}

// Successive randomized compression (Sec. II.C.1, Figs. random tensor and src): y ~ H x for
// every state of x with sketch dimension chi. The Khatri-Rao sketch columns are chi product
// states (bond one) whose node tensors are the columns c_k^(i) of Omega^(i); their top-down
// environments with H and x (pair s * chi + k) sketch everything outside an edge. Leaves to
// root: the local sketch Y_i[k][s_children][p] is the H_eff-type contraction of node i with the
// parent edge's down sketch (column index k as its bra bond) and the children's residual
// environments R_c = <y|H|x>; its QR over (s_children, p) x k gives the new node tensor (the
// identity when there are at most chi rows) and R_i; the root contracts directly. y's bonds
// are min(chi, d_i * prod of its children's bonds) and must be set on entry.
template <class T>
static void src_impl(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* x, int chi,
                     const std::vector<std::vector<double>>& omega, ttn_block* y) {
  const TreeInfo& tr = x->tree;
  const int n = x->n_states;
  cudaStream_t st = ctx->stream;
  if (n == 0) return;
  // the chi sketch columns as a block of product states
  ttn_block* skp = nullptr;
  {
    ttn_tree tmp;
    tmp.ctx = ctx;
    tmp.info = tr;
    std::vector<int> ones(tr.n, 1);
    ttn_status cs = ttn_block_create(ctx, &tmp, chi, ones.data(), &skp);
    if (cs != TTN_OK) TTN_FAIL(cs, "%s", ctx->last_error.c_str());
  }
  std::unique_ptr<ttn_block> sk(skp);
  for (int t = 0; t < tr.n; ++t) {
    const int d = tr.d(t);
    std::vector<double> h((size_t)chi * d, 1.0);
    if (tr.phys[t] > 0)
      for (int k = 0; k < chi; ++k)
        for (int p = 0; p < d; ++p) h[(size_t)k * d + p] = omega[t][(size_t)p * chi + k];
    CUDA_CHECK(cudaMemcpyAsync(sk->node64(t), h.data(), h.size() * sizeof(double),
                               cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
  }
  sk->touch();
  std::vector<int> pb((size_t)n * chi), pk((size_t)n * chi), id(n);
  for (int s = 0; s < n; ++s) {
    id[s] = s;
    for (int k = 0; k < chi; ++k) {
      pb[(size_t)s * chi + k] = k;
      pk[(size_t)s * chi + k] = s;
    }
  }
  EnvCache<T> sketch;
  sketch.init(ctx, H, sk.get(), x, pb, pk);
  DevVec did_b, did_k;
  PairSet ps = make_pairs(id, id, did_b, did_k, st);
  std::vector<DevBuf> R(tr.n);
  for (int t : tr.post) {
    const int nl = tr.nlegs(t);
    std::vector<const T*> env(nl, nullptr);
    std::vector<int> da(nl);
    const int off = t == tr.root ? 0 : 1;
    for (int m = off; m < nl; ++m) {
      const int c = tr.legs[t][m];
      env[m] = R[c].as<T>();
      da[m] = y->bond[c];
    }
    if (t == tr.root) {
      T* out = work_node<T>(y, t);
      node_op<T>(ctx, H, t, -1, nullptr, x, ps, env, da, out, (long long)n * y->size[t],
                 OUT_LOCAL);
      continue;
    }
    const int Dw = H->wbond[t], Db = x->bond[t];
    DevBuf E0((size_t)n * Dw * chi * Db * sizeof(T), st);
    {
      const int dims[4] = {n, chi, Dw, Db}, perm[4] = {0, 2, 1, 3};
      launch_permute<T>(ctx, sketch.get_down(t), E0.as<T>(), 1, 4, dims, perm);
    }
    env[0] = E0.as<T>();
    da[0] = chi;
    long long rows = tr.d(t);
    for (int m = 1; m < nl; ++m) rows *= da[m];
    DevBuf Y((size_t)n * chi * rows * sizeof(T), st);
    node_op<T>(ctx, H, t, -1, nullptr, x, ps, env, da, Y.p, (long long)n * chi * rows, OUT_LOCAL);
    T* node = work_node<T>(y, t);
    TTN_REQUIRE(y->size[t] == rows * y->bond[t], "src: output bonds do not match node %d", t);
    if (rows <= chi) {
      std::vector<T> eye((size_t)n * rows * rows, T(0));
      for (int s = 0; s < n; ++s)
        for (long long r = 0; r < rows; ++r) eye[(size_t)s * rows * rows + r * rows + r] = T(1);
      CUDA_CHECK(cudaMemcpyAsync(node, eye.data(), eye.size() * sizeof(T),
                                 cudaMemcpyHostToDevice, st));
      CUDA_CHECK(cudaStreamSynchronize(st));
    } else {
      TTN_REQUIRE(chi <= 64, "src: chi = %d above 64 is not supported", chi);
      const long long msz = rows * chi;
      DevBuf M((size_t)n * msz * sizeof(T), st), Q((size_t)n * msz * sizeof(T), st),
          Rq((size_t)n * chi * chi * sizeof(T), st);
      const int d1[2] = {chi, (int)rows}, p1[2] = {1, 0};
      launch_permute<T>(ctx, Y.as<T>(), M.as<T>(), n, 2, d1, p1);
      {
        LaunchScope ls(ctx, sizeof(T) == 8 ? "householder_qr_f64" : "householder_qr_f32",
                       4.0 * rows * chi * chi * n, 4.0 * sizeof(T) * msz * n);
        const size_t smem = 2 * (size_t)msz * sizeof(T);
        const bool on_chip = smem <= 200 * 1024;
        if (on_chip)
          CUDA_CHECK(cudaFuncSetAttribute(householder_qr_kernel<T>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        householder_qr_kernel<T><<<n, kT, on_chip ? smem : 0, st>>>(
            M.as<T>(), Q.as<T>(), Rq.as<T>(), (int)rows, chi, msz, on_chip ? 1 : 0);
        CUDA_LAUNCH_CHECK();
      }
      const int d2[2] = {(int)rows, chi}, p2[2] = {1, 0};
      launch_permute<T>(ctx, Q.as<T>(), node, n, 2, d2, p2);
    }
    std::vector<const T*> renv(nl, nullptr);
    for (int m = 1; m < nl; ++m) renv[m] = env[m];
    const long long esz = (long long)n * Dw * y->bond[t] * Db;
    R[t] = DevBuf((size_t)esz * sizeof(T), st);
    node_op<T>(ctx, H, t, 0, y, x, ps, renv, {}, R[t].p, esz, OUT_ENV);
  }
  commit<T>(y);
  CUDA_CHECK(cudaStreamSynchronize(st));
}

// Single-linkage blocks of the Rayleigh quotients (sorted values closer than `gap` join); gap <= 0
// gives one block per state.
static std::vector<std::vector<int>> clusters_by_gap(const std::vector<double>& lam, double gap) {
  const int n = (int)lam.size();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  std::vector<std::vector<int>> out;
  for (int k = 0; k < n; ++k) {
    if (k > 0 && gap > 0.0 && lam[order[k]] - lam[order[k - 1]] < gap) out.back().push_back(order[k]);
    else out.push_back({order[k]});
  }
  for (auto& c : out) std::sort(c.begin(), c.end());
  return out;
}

// Rayleigh-Ritz over the states of Y and refit (the orthogonalisation step of Alg. 3, and the
// generalized eigenvalue problem Hc = ESc of Sec. III.B over a whole block): H~ and M~ over Y,
// canonical orthogonalisation (eigenvalues of M~ below rr_eps * max dropped), X_a = the fitted
// sum_b v_ba Y_b of the a-th Ritz vector (fit starts from the Y_b of largest |v_ba|),
// normalised. theta receives the Ritz values; X and Y hold the same number of states.
template <class T>
static void rr_refit(ttn_ctx* ctx, ttn_ttno* H, ttn_ttno* Id, const ttn_block* Y, ttn_block* X,
                     double rr_eps, int fit_sweeps, int prec, std::vector<double>& theta) {
  cudaStream_t st = ctx->stream;
  const int m = Y->n_states;
  DevBuf Ht((size_t)m * m * sizeof(double), st), Mt((size_t)m * m * sizeof(double), st),
      th((size_t)m * sizeof(double), st), V((size_t)m * m * sizeof(double), st);
  CUDA_CHECK(cudaMemsetAsync(Ht.p, 0, (size_t)m * m * sizeof(double), st));
  CUDA_CHECK(cudaMemsetAsync(Mt.p, 0, (size_t)m * m * sizeof(double), st));
  if (gram_device(ctx, H, Y, Y, Ht.as<double>(), m, prec) +
      gram_device(ctx, Id, Y, Y, Mt.as<double>(), m, prec))
    TTN_FAIL(TTN_ENONFINITE, "Rayleigh-Ritz of a block: non-finite Gram entries");
  rayleigh_ritz_device(ctx, m, Ht.as<double>(), Mt.as<double>(), m, rr_eps, th.as<double>(),
                       V.as<double>());
  std::vector<double> hV((size_t)m * m);
  theta.assign(m, 0.0);
  CUDA_CHECK(cudaMemcpyAsync(theta.data(), th.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaMemcpyAsync(hV.data(), V.p, hV.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  FitGroup g{Id, Y, {}, {}, {}};
  std::vector<int> init(m);
  for (int a = 0; a < m; ++a) {
    int arg = 0;
    double best = -1.0;
    for (int b = 0; b < m; ++b) {
      const double v = hV[(size_t)b * m + a];
      if (std::fabs(v) > best) {
        best = std::fabs(v);
        arg = b;
      }
      if (v != 0.0) {
        g.out_j.push_back(a);
        g.in_k.push_back(b);
        g.coef.push_back(v);
      }
    }
    init[a] = arg;
  }
  ttn_status cs = ttn_block_copy_states(X, Y, m, init.data());
  if (cs != TTN_OK) TTN_FAIL(cs, "copy");
  std::vector<FitGroup> gs{g};
  fit_impl<T>(ctx, gs, X, fit_sweeps);
  normalize_states<T>(ctx, X, prec);
}

// Block inverse iteration (Alg. 3): every block uses the mean Rayleigh quotient of its states as
// the shift; every state is solved by ALS; blocks of more than one state are re-orthogonalised
// by their own Rayleigh-Ritz step and refitted.
template <class T>
static void inverse_iteration_impl(ttn_ctx* ctx, ttn_ttno* H, ttn_block* x, int n_iter,
                                   double gap, int als_sweeps, int mr_max, double mr_tol,
                                   int fit_sweeps, int prec, double* eig_hist, bool& hit) {
  const TreeInfo& tr = x->tree;
  const int n = x->n_states;
  cudaStream_t st = ctx->stream;
  ttn_ttno* Id = identity_for(ctx, tr);
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  auto new_block = [&](int ns) {
    ttn_tree tmp;
    tmp.ctx = ctx;
    tmp.info = tr;
    ttn_block* b = nullptr;
    ttn_status s = ttn_block_create(ctx, &tmp, ns, x->bond.data(), &b);
    if (s != TTN_OK) TTN_FAIL(s, "%s", ctx->last_error.c_str());
    return std::unique_ptr<ttn_block>(b);
  };
  auto diag = [&](ttn_ttno* op, const ttn_block* b) {
    DevBuf dv((size_t)n * sizeof(double), st);
    gram_pairs<T>(ctx, op, b, b, id, id, dv.as<double>());
    std::vector<double> h(n);
    CUDA_CHECK(cudaMemcpyAsync(h.data(), dv.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    return h;
  };
  iter_clock_start(ctx);
  normalize_states<T>(ctx, x, prec);
  std::vector<double> lam = diag(H, x);
  if (eig_hist) std::copy(lam.begin(), lam.end(), eig_hist);
  iter_clock_mark(ctx);
  auto Y = new_block(n), Xn = new_block(n);
  const double rr_eps = prec == TTN_FP64 ? 1e-12 : 1e-6;
  for (int it = 1; it <= n_iter; ++it) {
    const auto blocks = clusters_by_gap(lam, gap);
    std::vector<double> shift(n);
    for (const auto& c : blocks) {
      double m = 0.0;
      for (int j : c) m += lam[j];
      for (int j : c) shift[j] = m / c.size();
    }
    {
      PhaseScope ph(ctx, "als_inverse");
      ttn_status cs = ttn_block_copy_states(Y.get(), x, n, id.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      hit |= als_impl<T>(ctx, H, shift, x, Y.get(), als_sweeps, mr_max, mr_tol);
      normalize_states<T>(ctx, Y.get(), prec);
    }
    std::vector<double> lam_n = diag(H, Y.get());
    {
      ttn_status cs = ttn_block_copy_states(Xn.get(), Y.get(), n, id.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
    }
    for (const auto& c : blocks) {
      const int m = (int)c.size();
      if (m == 1) continue;
      PhaseScope ph(ctx, "block_rayleigh_ritz");
      auto Yc = new_block(m), Xc = new_block(m);
      ttn_status cs = ttn_block_copy_states(Yc.get(), Y.get(), m, c.data());
      if (cs != TTN_OK) TTN_FAIL(cs, "copy");
      std::vector<double> hth;
      rr_refit<T>(ctx, H, Id, Yc.get(), Xc.get(), rr_eps, fit_sweeps, prec, hth);
      for (int a = 0; a < m; ++a) {
        lam_n[c[a]] = hth[a];
        for (int t = 0; t < tr.n; ++t)
          CUDA_CHECK(cudaMemcpyAsync(Xn->node64(t) + (long long)c[a] * Xn->size[t],
                                     Xc->node64(t) + (long long)a * Xc->size[t],
                                     Xn->size[t] * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
      Xn->touch();
    }
    ttn_status cs = ttn_block_copy_states(x, Xn.get(), n, id.data());
    if (cs != TTN_OK) TTN_FAIL(cs, "copy");
    lam = lam_n;
    if (eig_hist) std::copy(lam.begin(), lam.end(), eig_hist + (size_t)it * n);
    iter_clock_mark(ctx);
  }
  CUDA_CHECK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------------------------------------
// Rayleigh-Ritz without device allocation.
//
// Some callers may not allocate device memory once they are running: a serving process that
// reserves its device budget at start-up, a memory pool that is frozen after initialisation, a
// host framework that owns the allocator. For them ttn_rayleigh_ritz_noalloc works in a fixed
// working area that lives for the life of the process: the file-scope array below. Its size
// bounds the problem (m <= TTN_RR_NOALLOC_MAX_M); every GPU that loads the library holds it
// until exit.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr int kRRMaxM = TTN_RR_NOALLOC_MAX_M;
// A, U, Us, X, HX, Hp, Y (m x m each) + mu, th (m each) + keep indices (m ints, stored in m
// doubles) + the final off-diagonal ratios of the two Jacobi solves (padded to 8 doubles)
constexpr size_t kRRScratchDoubles = 7ull * kRRMaxM * kRRMaxM + 3ull * kRRMaxM + 8;
// A Jacobi solve whose final sqrt(off-diagonal / total) is above this did not converge.
constexpr double kRRJacobiOffBound = 1e-10;
static __device__ __align__(256) double g_rr_scratch[kRRScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_rr_scratch_dev[kMaxDevices] = {nullptr};
std::once_flag g_rr_once[kMaxDevices];
cudaError_t g_rr_setup_err[kMaxDevices] = {cudaSuccess};

// Device address of the working area on `device` (which must be current), and the kernels of
// the no-allocation call loaded: under lazy module loading a kernel's code is loaded, and device
// memory taken for it, at its first launch, which must not happen inside a no-allocation call.
// Done once per device, when a context is created on it (and, failing that, at the first call);
// the host-side name of a __device__ array is only a stand-in, so the address has to come from
// cudaGetSymbolAddress.
double* rr_scratch_for(int device) {
  TTN_REQUIRE(device >= 0 && device < kMaxDevices, "device %d out of range", device);
  std::call_once(g_rr_once[device], [device] {
    void* p = nullptr;
    g_rr_setup_err[device] = cudaGetSymbolAddress(&p, g_rr_scratch);
    if (g_rr_setup_err[device] == cudaSuccess) g_rr_scratch_dev[device] = static_cast<double*>(p);
    const void* kernels[] = {(const void*)symmetrize_kernel, (const void*)jacobi_kernel,
                             (const void*)sort_eig_kernel, (const void*)canon_basis_kernel,
                             (const void*)small_gemm_kernel, (const void*)fix_sign_kernel};
    for (const void* k : kernels) {
      cudaFuncAttributes fa;
      if (g_rr_setup_err[device] == cudaSuccess)
        g_rr_setup_err[device] = cudaFuncGetAttributes(&fa, k);
    }
  });
  if (g_rr_setup_err[device] != cudaSuccess)
    TTN_FAIL(TTN_ECUDA, "cudaGetSymbolAddress of the Rayleigh-Ritz working area failed: %s",
             cudaGetErrorString(g_rr_setup_err[device]));
  return g_rr_scratch_dev[device];
}

}  // namespace

// Called when a context is created on `device` (current): prepares the no-allocation
// Rayleigh-Ritz there (working-area address, its kernels loaded).
void rr_noalloc_prepare(int device) { rr_scratch_for(device); }

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

ttn_status ttn_recompress(ttn_ctx* ctx, int n_in, const double* coeff, const ttn_ttno* const* ops,
                          const ttn_block* const* in, const int* in_state, ttn_block* out,
                          int n_out, int n_sweeps, ttn_precision prec) {
  if (!ctx || !out) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    TTN_REQUIRE(n_in >= 0 && (n_in == 0 || (coeff && ops && in && in_state)), "inputs");
    TTN_REQUIRE(n_out == out->n_states, "n_out must equal the states of `out`");
    TTN_REQUIRE(n_sweeps >= 0, "n_sweeps < 0");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    std::vector<FitGroup> groups;
    for (int k = 0; k < n_in; ++k) {
      check_block_like(in[k], out);
      TTN_REQUIRE(in_state[k] >= 0 && in_state[k] < in[k]->n_states, "in_state[%d]", k);
      ttn_ttno* op = ops[k] ? const_cast<ttn_ttno*>(ops[k]) : identity_for(ctx, out->tree);
      if (ops[k]) TTN_REQUIRE(op->tree.same_shape(out->tree), "operator %d: other tree", k);
      size_t g = 0;
      for (; g < groups.size(); ++g)
        if (groups[g].op == op && groups[g].in == in[k]) break;
      if (g == groups.size()) groups.push_back({op, in[k], {}, {}, {}});
    }
    for (auto& g : groups) {
      for (int j = 0; j < n_out; ++j)
        for (int k = 0; k < n_in; ++k) {
          ttn_ttno* op = ops[k] ? const_cast<ttn_ttno*>(ops[k]) : identity_for(ctx, out->tree);
          const double c = coeff[(size_t)k * n_out + j];
          if (op == g.op && in[k] == g.in && c != 0.0) {
            g.out_j.push_back(j);
            g.in_k.push_back(in_state[k]);
            g.coef.push_back(c);
          }
        }
    }
    if (prec == TTN_FP64) fit_impl<double>(ctx, groups, out, n_sweeps);
    else fit_impl<float>(ctx, groups, out, n_sweeps);
    return TTN_OK;
  });
}

ttn_status ttn_als_solve(ttn_ctx* ctx, const ttn_ttno* H, const double* shift,
                         const ttn_block* rhs, ttn_block* y, int n_sweeps, int minres_max,
                         double minres_tol, ttn_precision prec) {
  if (!ctx || !H || !shift || !rhs || !y) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    check_block_like(rhs, y);
    TTN_REQUIRE(rhs->n_states == y->n_states, "rhs and y differ in state count");
    TTN_REQUIRE(H->tree.same_shape(y->tree), "operator on another tree");
    TTN_REQUIRE(n_sweeps >= 0 && minres_max >= 0 && minres_tol >= 0.0, "bad solver settings");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    std::vector<double> s(shift, shift + y->n_states);
    bool hit = prec == TTN_FP64
                   ? als_impl<double>(ctx, const_cast<ttn_ttno*>(H), s, rhs, y, n_sweeps,
                                      minres_max, minres_tol)
                   : als_impl<float>(ctx, const_cast<ttn_ttno*>(H), s, rhs, y, n_sweeps,
                                     minres_max, minres_tol);
    if (!hit) return TTN_OK;
    ctx->last_error = "a local MINRES solve reached minres_max before its tolerance (results "
                      "written)";
    return TTN_ENOTCONV;
  });
}

ttn_status ttn_rayleigh_ritz(ttn_ctx* ctx, int m, const double* Ht, const double* Mt, int n,
                             double eps, double* theta, double* V) {
  if (!ctx || !Ht || !Mt || !theta || !V) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    TTN_REQUIRE(m >= 1 && n >= 1 && n <= m, "need 1 <= n <= m");
    cudaStream_t st = ctx->stream;
    const size_t mm = (size_t)m * m;
    DevBuf dH(mm * sizeof(double), st), dM(mm * sizeof(double), st), dth(n * sizeof(double), st),
        dV((size_t)m * n * sizeof(double), st);
    CUDA_CHECK(cudaMemcpyAsync(dH.p, Ht, mm * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(dM.p, Mt, mm * sizeof(double), cudaMemcpyHostToDevice, st));
    rayleigh_ritz_device(ctx, m, dH.as<double>(), dM.as<double>(), n, eps, dth.as<double>(),
                         dV.as<double>());
    CUDA_CHECK(cudaMemcpyAsync(theta, dth.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(V, dV.p, (size_t)m * n * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    return TTN_OK;
  });
}

ttn_status ttn_lobpcg(ttn_ctx* ctx, const ttn_ttno* H, ttn_block* x, int n_iter,
                      double shift_offset, int als_sweeps, int minres_max, double minres_tol,
                      int fit_sweeps, ttn_precision prec, double* eig_hist) {
  if (!ctx || !H || !x) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    TTN_REQUIRE(n_iter >= 0 && als_sweeps >= 0 && minres_max >= 0 && fit_sweeps >= 0,
                "bad solver settings");
    TTN_REQUIRE(x->n_states >= 1, "empty block");
    TTN_REQUIRE(H->tree.same_shape(x->tree), "operator on another tree");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    bool hit = false;
    if (prec == TTN_FP64)
      lobpcg_impl<double>(ctx, const_cast<ttn_ttno*>(H), x, n_iter, shift_offset, als_sweeps,
                          minres_max, minres_tol, fit_sweeps, prec, eig_hist, hit);
    else
      lobpcg_impl<float>(ctx, const_cast<ttn_ttno*>(H), x, n_iter, shift_offset, als_sweeps,
                         minres_max, minres_tol, fit_sweeps, prec, eig_hist, hit);
    if (!hit) return TTN_OK;
    ctx->last_error = "a local MINRES solve reached minres_max before its tolerance (results "
                      "written)";
    return TTN_ENOTCONV;
  });
}

ttn_status ttn_inverse_iteration(ttn_ctx* ctx, const ttn_ttno* H, ttn_block* x, int n_iter,
                                 double cluster_gap, int als_sweeps, int minres_max,
                                 double minres_tol, int fit_sweeps, ttn_precision prec,
                                 double* rq_hist) {
  if (!ctx || !H || !x) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    TTN_REQUIRE(n_iter >= 0 && als_sweeps >= 0 && minres_max >= 0 && fit_sweeps >= 0,
                "bad solver settings");
    TTN_REQUIRE(x->n_states >= 1, "empty block");
    TTN_REQUIRE(H->tree.same_shape(x->tree), "operator on another tree");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    bool hit = false;
    if (prec == TTN_FP64)
      inverse_iteration_impl<double>(ctx, const_cast<ttn_ttno*>(H), x, n_iter, cluster_gap,
                                     als_sweeps, minres_max, minres_tol, fit_sweeps, prec,
                                     rq_hist, hit);
    else
      inverse_iteration_impl<float>(ctx, const_cast<ttn_ttno*>(H), x, n_iter, cluster_gap,
                                    als_sweeps, minres_max, minres_tol, fit_sweeps, prec,
                                    rq_hist, hit);
    if (!hit) return TTN_OK;
    ctx->last_error = "a local MINRES solve reached minres_max before its tolerance (results "
                      "written)";
    return TTN_ENOTCONV;
  });
}

ttn_status ttn_block_rayleigh_ritz(ttn_ctx* ctx, const ttn_ttno* Hc, ttn_block* x, double eps,
                                   int fit_sweeps, ttn_precision prec, double* theta) {
  if (!ctx || !Hc || !x) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    ttn_ttno* H = const_cast<ttn_ttno*>(Hc);
    TTN_REQUIRE(H->tree.same_shape(x->tree), "operator on another tree");
    TTN_REQUIRE(x->n_states >= 1 && fit_sweeps >= 1 && eps >= 0.0, "bad arguments");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    ttn_ttno* Id = identity_for(ctx, x->tree);
    ttn_block* yb = nullptr;
    {
      ttn_tree tmp;
      tmp.ctx = ctx;
      tmp.info = x->tree;
      ttn_status cs = ttn_block_create(ctx, &tmp, x->n_states, x->bond.data(), &yb);
      if (cs != TTN_OK) TTN_FAIL(cs, "%s", ctx->last_error.c_str());
    }
    std::unique_ptr<ttn_block> Y(yb);
    std::vector<int> id(x->n_states);
    std::iota(id.begin(), id.end(), 0);
    ttn_status cs = ttn_block_copy_states(Y.get(), x, x->n_states, id.data());
    if (cs != TTN_OK) TTN_FAIL(cs, "copy");
    std::vector<double> th;
    if (prec == TTN_FP64) rr_refit<double>(ctx, H, Id, Y.get(), x, eps, fit_sweeps, prec, th);
    else rr_refit<float>(ctx, H, Id, Y.get(), x, eps, fit_sweeps, prec, th);
    if (theta) std::copy(th.begin(), th.end(), theta);
    return TTN_OK;
  });
}

ttn_status ttn_src_apply(ttn_ctx* ctx, const ttn_ttno* Hc, const ttn_block* x, int chi,
                         const double* omega, ttn_block** out, ttn_precision prec) {
  if (!ctx || !Hc || !x || !omega || !out) return TTN_EINVAL;
  *out = nullptr;
  return guarded_s(ctx, [&]() -> ttn_status {
    PrecisionScope prec_scope(ctx, prec);
    ttn_ttno* H = const_cast<ttn_ttno*>(Hc);
    const TreeInfo& tr = x->tree;
    TTN_REQUIRE(H->tree.same_shape(tr), "TTNO and block live on different trees");
    TTN_REQUIRE(chi >= 1 && chi <= 64, "chi = %d outside [1, 64]", chi);
    TTN_REQUIRE(valid_precision(prec),
                "unknown precision %d", (int)prec);
    std::vector<std::vector<double>> om(tr.n);
    long long o = 0;
    for (int t = 0; t < tr.n; ++t) {
      if (tr.phys[t] <= 0) continue;
      om[t].assign(omega + o, omega + o + (long long)tr.phys[t] * chi);
      o += (long long)tr.phys[t] * chi;
    }
    for (long long i = 0; i < o; ++i)
      if (!std::isfinite(omega[i])) TTN_FAIL(TTN_ENONFINITE, "omega[%lld] is not finite", i);
    std::vector<int> bond(tr.n, 1);
    for (int t : tr.post) {
      if (t == tr.root) continue;
      long long rows = tr.d(t);
      for (int c : tr.children[t]) rows *= bond[c];
      bond[t] = (int)std::min<long long>(chi, rows);
    }
    ttn_block* yb = nullptr;
    {
      ttn_tree tmp;
      tmp.ctx = ctx;
      tmp.info = tr;
      ttn_status cs = ttn_block_create(ctx, &tmp, x->n_states, bond.data(), &yb);
      if (cs != TTN_OK) TTN_FAIL(cs, "%s", ctx->last_error.c_str());
    }
    std::unique_ptr<ttn_block> guard(yb);
    if (prec == TTN_FP64) src_impl<double>(ctx, H, x, chi, om, yb);
    else src_impl<float>(ctx, H, x, chi, om, yb);
    *out = guard.release();
    return TTN_OK;
  });
}

ttn_status ttn_rayleigh_ritz_noalloc(ttn_ctx* ctx, int m, const double* Ht, const double* Mt,
                                     int n, double eps, double* theta, double* V) {
  if (!ctx || !Ht || !Mt || !theta || !V) return TTN_EINVAL;
  return guarded_s(ctx, [&]() -> ttn_status {
    TTN_REQUIRE(ctx->device >= 0, "a host-only context has no device");
    TTN_REQUIRE(m >= 1 && n >= 1 && n <= m, "need 1 <= n <= m (m = %d, n = %d)", m, n);
    TTN_REQUIRE(m <= kRRMaxM,
                "m = %d exceeds the no-allocation limit TTN_RR_NOALLOC_MAX_M = %d; use "
                "ttn_rayleigh_ritz", m, kRRMaxM);
    int prev_device = -1;
    CUDA_CHECK(cudaGetDevice(&prev_device));
    struct Restore {
      int d;
      ~Restore() {
        if (d >= 0) cudaSetDevice(d);
      }
    } restore{prev_device};
    CUDA_CHECK(cudaSetDevice(ctx->device));
    double* base = rr_scratch_for(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t mm = (size_t)m * m;
    double* A = base;
    double* U = A + mm;
    double* Us = U + mm;
    double* X = Us + mm;
    double* HX = X + mm;
    double* Hp = HX + mm;
    double* Y = Hp + mm;
    double* mu = Y + mm;
    double* th = mu + m;
    int* keep = reinterpret_cast<int*>(th + m);
    double* offr = th + 2 * m;
    auto eig = [&](double* Ain, int k, double* evals, double* Vout, double* off_out) {
      symmetrize_kernel<<<grid_of((long long)k * k), kT, 0, st>>>(Ain, k);
      const int kp = k + (k & 1);
      const size_t sh = (size_t)kp * sizeof(double) + (size_t)kp * sizeof(int) + 64;
      jacobi_kernel<<<1, 1024, sh, st>>>(Ain, U, k, 40, 1e-15, off_out);
      sort_eig_kernel<<<1, 256, k * sizeof(int), st>>>(Ain, U, k, evals, Vout);
      ctx->launches += 3;
      CUDA_LAUNCH_CHECK();
    };
    CUDA_CHECK(cudaMemcpyAsync(A, Mt, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
    eig(A, m, mu, Us, offr);
    double hmu[kRRMaxM];
    double hoff[2] = {0.0, 0.0};
    CUDA_CHECK(cudaMemcpyAsync(hmu, mu, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(hoff, offr, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    double mx = hmu[0];
    for (int i = 0; i < m; ++i) {
      if (!std::isfinite(hmu[i])) TTN_FAIL(TTN_ENONFINITE, "non-finite overlap matrix");
      mx = std::max(mx, hmu[i]);
    }
    int hkeep[kRRMaxM];
    int k = 0;
    for (int i = 0; i < m; ++i)
      if (hmu[i] > eps * mx) hkeep[k++] = i;
    TTN_REQUIRE(k >= n, "only %d of %d directions survive eps = %g", k, n, eps);
    CUDA_CHECK(cudaMemcpyAsync(keep, hkeep, k * sizeof(int), cudaMemcpyHostToDevice, st));
    canon_basis_kernel<<<grid_of((long long)m * k), kT, 0, st>>>(Us, mu, keep, m, k, X);
    small_gemm_kernel<<<grid_of((long long)m * k), kT, 0, st>>>(Ht, m, 1, X, k, 1, HX, m, k, m);
    small_gemm_kernel<<<grid_of((long long)k * k), kT, 0, st>>>(X, 1, k, HX, k, 1, Hp, k, k, m);
    ctx->launches += 3;
    CUDA_LAUNCH_CHECK();
    eig(Hp, k, th, Y, offr + 1);
    small_gemm_kernel<<<grid_of((long long)m * n), kT, 0, st>>>(X, k, 1, Y, k, 1, V, m, n, k);
    fix_sign_kernel<<<(n + 127) / 128, 128, 0, st>>>(V, m, n);
    ctx->launches += 2;
    CUDA_LAUNCH_CHECK();
    CUDA_CHECK(cudaMemcpyAsync(theta, th, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(hoff + 1, offr + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    if (!(hoff[0] <= kRRJacobiOffBound && hoff[1] <= kRRJacobiOffBound)) {
      ctx->last_error = ttn_fmt("Jacobi eigensolver stopped at off-diagonal ratios %.3g (overlap) "
                                "and %.3g (projected H), above %.0e (results written)",
                                hoff[0], hoff[1], kRRJacobiOffBound);
      return TTN_ENOTCONV;
    }
    return TTN_OK;
  });
}

}  // extern "C"
