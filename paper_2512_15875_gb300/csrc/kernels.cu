// Generic device kernels of the contraction engine: a strided batched GEMM with per-item
// segment sums (the workhorse of every node contraction), tensor permutes, per-pair dots.
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <set>

#include <cuda.h>

#include "internal.h"

namespace {

constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ const T* operand_base(const GemmOperand& o, int pair, const int* pb,
                                                 const int* pk) {
  long long idx = 0;
  if (o.mode == MODE_PAIR) idx = pair;
  else if (o.mode == MODE_BRA) idx = pb[pair];
  else if (o.mode == MODE_KET) idx = pk[pair];
  return static_cast<const T*>(o.base) + idx * o.pstride;
}

// One CTA computes a BM x BN tile of one item (pair, sub) of
//   C[item](m, n) = sum_{segments s of sub} sum_k A_s(m, k) * B_s(n, k)
// with arbitrary element strides. Shared-memory tiles are stored k-major; each thread owns a
// TM x TN register tile with rows/columns strided by BM/TM and BN/TN (conflict-free reads).
template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads) gemm_kernel(GemmDesc g, int tiles_m, int tiles_n) {
  static_assert((BM / TM) * (BN / TN) == kThreads, "tile/thread mismatch");
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const long long tiles = (long long)tiles_m * tiles_n;
  const long long bid = blockIdx.x;
  const int tile = (int)(bid % tiles);
  const long long rest = bid / tiles;
  const int sub = (int)(rest % g.st.n_sub);
  const int pair = (int)(rest / g.st.n_sub);
  const int m0 = (tile / tiles_n) * BM;
  const int n0 = (tile % tiles_n) * BN;
  const T* Ab = operand_base<T>(g.A, pair, g.pair_bra, g.pair_ket);
  const T* Bb = operand_base<T>(g.B, pair, g.pair_bra, g.pair_ket);
  const int tid = threadIdx.x;
  const int ty = tid / (BN / TN), tx = tid % (BN / TN);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  const int s_begin = g.st.seg_ptr[sub], s_end = g.st.seg_ptr[sub + 1];
  for (int s = s_begin; s < s_end; ++s) {
    const T* Ap = Ab + g.st.seg_a[s];
    const T* Bp = Bb + g.st.seg_b[s];
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      if (g.a_sm == 1) {
        for (int i = tid; i < BM * BK; i += kThreads) {
          const int m = i % BM, k = i / BM, gm = m0 + m, gk = k0 + k;
          As[k][m] = (gm < g.M && gk < g.K) ? Ap[gm + (long long)gk * g.a_sk] : T(0);
        }
      } else {
        for (int i = tid; i < BM * BK; i += kThreads) {
          const int k = i % BK, m = i / BK, gm = m0 + m, gk = k0 + k;
          As[k][m] = (gm < g.M && gk < g.K) ? Ap[(long long)gm * g.a_sm + (long long)gk * g.a_sk]
                                            : T(0);
        }
      }
      if (g.b_sn == 1) {
        for (int i = tid; i < BN * BK; i += kThreads) {
          const int n = i % BN, k = i / BN, gn = n0 + n, gk = k0 + k;
          Bs[k][n] = (gn < g.N && gk < g.K) ? Bp[gn + (long long)gk * g.b_sk] : T(0);
        }
      } else {
        for (int i = tid; i < BN * BK; i += kThreads) {
          const int k = i % BK, n = i / BK, gn = n0 + n, gk = k0 + k;
          Bs[k][n] = (gn < g.N && gk < g.K) ? Bp[(long long)gn * g.b_sn + (long long)gk * g.b_sk]
                                            : T(0);
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[k][ty + i * (BM / TM)];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx + j * (BN / TN)];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  T* Cb = static_cast<T*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * (BM / TM);
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * (BN / TN);
      if (gn < g.N) Cb[(long long)gm * g.c_sm + (long long)gn * g.c_sn] = acc[i][j];
    }
  }
}

struct TileCfg {
  int bm, bn;
};
constexpr TileCfg kCfgs[] = {{64, 64}, {64, 32}, {32, 32}, {128, 16}, {64, 16}, {16, 16}};

template <class T>
void dispatch(int cfg, const GemmDesc& g, int tm, int tn, long long grid, cudaStream_t s) {
  switch (cfg) {
    case 0: gemm_kernel<T, 64, 64, 16, 4, 4><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
    case 1: gemm_kernel<T, 64, 32, 16, 4, 2><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
    case 2: gemm_kernel<T, 32, 32, 16, 2, 2><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
    case 3: gemm_kernel<T, 128, 16, 16, 8, 1><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
    case 4: gemm_kernel<T, 64, 16, 16, 4, 1><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
    default: gemm_kernel<T, 16, 16, 16, 1, 1><<<grid, kThreads, 0, s>>>(g, tm, tn); break;
  }
}

struct PermArgs {
  int nd;
  long long od[8];   // output dims
  long long is[8];   // input stride of the input axis placed at each output position
};

template <class T>
__global__ void permute_kernel(const T* __restrict__ in, T* __restrict__ out, long long batch,
                               long long size, PermArgs a) {
  const long long total = batch * size;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / size;
    long long r = idx - b * size, src = 0;
    for (int k = a.nd - 1; k >= 0; --k) {
      const long long c = r % a.od[k];
      r /= a.od[k];
      src += c * a.is[k];
    }
    out[idx] = in[b * size + src];
  }
}

template <class T>
__global__ void pair_dot_kernel(const T* __restrict__ bra, long long bra_stride,
                                const T* __restrict__ Z, long long z_stride, long long n,
                                const int* __restrict__ pb, double* __restrict__ out) {
  const int pair = blockIdx.x;
  const T* a = bra + (long long)pb[pair] * bra_stride;
  const T* z = Z + (long long)pair * z_stride;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += (double)a[i] * (double)z[i];
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[pair] = acc;
  }
}

template <class T>
__global__ void shift_axpy_kernel(T* __restrict__ y, const T* __restrict__ x,
                                  const double* __restrict__ shift, long long size,
                                  long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / size;
    y[i] = y[i] - (T)shift[s] * x[i];
  }
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                              long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void to_f64_kernel(const float* __restrict__ in, double* __restrict__ out,
                              long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

__global__ void scatter_gram_kernel(const double* __restrict__ g, int n_pairs,
                                    const int* __restrict__ pb, const int* __restrict__ pk,
                                    int symmetric, double* __restrict__ out, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pairs) return;
  out[(long long)pb[i] * ld + pk[i]] = g[i];
  if (symmetric) out[(long long)pk[i] * ld + pb[i]] = g[i];
}

__global__ void count_nonfinite_kernel(const double* __restrict__ a, int rows, int cols, int ld,
                                       unsigned* __restrict__ count) {
  const long long total = (long long)rows * cols;
  unsigned c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    c += isfinite(a[(i / cols) * ld + i % cols]) ? 0u : 1u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// dst[j][r] = src[idx[j]][r] for j < n_rows, r < size (rows of `size` doubles)
__global__ void gather_rows_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                   const int* __restrict__ idx, long long size, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / size;
    dst[i] = src[(long long)idx[j] * size + (i - j * size)];
  }
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// Raises a kernel's dynamic shared-memory limit once per (kernel, device).
static void smem_attr(const void* fn, int bytes, int device) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, device})) return;
  CUDA_CHECK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({fn, device});
}

// 2-D tensor maps for the tensor copies (cp.async.bulk.tensor) of row blocks: a buffer of float
// rows, `row_len` elements per row, viewed as (row_len, rows); one box is box_x elements of
// box_y consecutive rows, landing densely in shared memory. The encoder is the driver's
// cuTensorMapEncodeTiled, reached through the runtime's entry-point query (no driver library
// link). Returns false where the buffer cannot be described (alignment, sizes).
using TensorMapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                       const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                       const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion,
                                       CUtensorMapFloatOOBfill);
static TensorMapEncodeFn tensor_map_encoder() {
  static TensorMapEncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<TensorMapEncodeFn>(p);
  }();
  return fn;
}
static bool make_row_tensor_map(CUtensorMap* m, const void* base, long long row_len, long long rows,
                                int box_x, int box_y) {
  const TensorMapEncodeFn enc = tensor_map_encoder();
  if (!enc || reinterpret_cast<uintptr_t>(base) % 16 || row_len <= 0 || rows <= 0 ||
      (row_len * 4) % 16 || box_x <= 0 || box_x > 256 || (box_x * 4) % 16 || box_y <= 0 ||
      box_y > 256 || row_len >= (1LL << 31) || rows >= (1LL << 31))
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)row_len, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)row_len * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Algorithmic bytes of a strided batched launch: the operands that are node tensors,
// environments or results of the contraction (GemmDesc::alg_*), every distinct slice once per
// distinct base (pair / bra / ket index); intermediates of the contraction chain (T_l, Z)
// count nothing.
static double algorithmic_bytes(const GemmDesc& g, size_t elem) {
  double n_ua = (double)g.hst->n_ua, n_ub = (double)g.hst->n_ub;
  if (g.hst->n_ua < 0 || g.hst->n_ub < 0) {
    n_ua = (double)std::set<long long>(g.hst->seg_a.begin(), g.hst->seg_a.end()).size();
    n_ub = (double)std::set<long long>(g.hst->seg_b.begin(), g.hst->seg_b.end()).size();
  }
  auto bases = [&](int mode) -> double {
    if (mode == MODE_PAIR) return g.n_pairs;
    if (mode == MODE_BRA) return std::min(g.n_pairs, g.max_bra + 1);
    if (mode == MODE_KET) return std::min(g.n_pairs, g.max_ket + 1);
    return 1.0;
  };
  const double a = g.alg_a ? bases(g.A.mode) * n_ua * g.M * g.K : 0.0;
  const double b = g.alg_b ? bases(g.B.mode) * n_ub * g.N * g.K : 0.0;
  const double c = g.alg_c ? (double)g.n_pairs * g.st.n_sub * g.M * g.N : 0.0;
  return (double)elem * (a + b + c);
}

// Host-side proof that every address the launch can form lies inside its buffer: for each item
// and segment, the smallest and largest offsets over (m, n, k) and over all pairs.
static void check_bounds(const GemmDesc& g, size_t elem) {
  auto base_max = [&](int mode, long long pstride) -> long long {
    if (mode == MODE_PAIR) return (long long)(g.n_pairs - 1) * pstride;
    if (mode == MODE_BRA) return (long long)g.max_bra * pstride;
    if (mode == MODE_KET) return (long long)g.max_ket * pstride;
    return 0;
  };
  TTN_REQUIRE(g.hst && (int)g.hst->sub_c.size() == g.st.n_sub, "gemm: missing host tables");
  const long long a_hi = base_max(g.A.mode, g.A.pstride) + (long long)(g.M - 1) * g.a_sm +
                         (long long)(g.K - 1) * g.a_sk;
  const long long b_hi = base_max(g.B.mode, g.B.pstride) + (long long)(g.N - 1) * g.b_sn +
                         (long long)(g.K - 1) * g.b_sk;
  const long long c_hi = base_max(g.c_mode, g.c_pstride) + (long long)(g.M - 1) * g.c_sm +
                         (long long)(g.N - 1) * g.c_sn;
  for (int s = 0; s < g.st.n_sub; ++s) {
    const long long c0 = g.hst->sub_c[s];
    if (c0 < 0 || c0 + c_hi >= g.c_len)
      TTN_FAIL(TTN_EINVAL, "gemm bounds: C item %d reaches %lld of %lld (elem %zu)", s, c0 + c_hi,
               g.c_len, elem);
    if (g.K <= 0) continue;
    for (int q = g.hst->seg_ptr[s]; q < g.hst->seg_ptr[s + 1]; ++q) {
      const long long a0 = g.hst->seg_a[q], b0 = g.hst->seg_b[q];
      if (a0 < 0 || a0 + a_hi >= g.a_len)
        TTN_FAIL(TTN_EINVAL, "gemm bounds: A seg %d reaches %lld of %lld", q, a0 + a_hi,
                 g.a_len);
      if (b0 < 0 || b0 + b_hi >= g.b_len)
        TTN_FAIL(TTN_EINVAL, "gemm bounds: B seg %d reaches %lld of %lld", q, b0 + b_hi,
                 g.b_len);
    }
  }
}

static cudaEvent_t pool_event(ttn_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CUDA_CHECK(cudaEventCreate(&e));
  return e;
}

LaunchScope::LaunchScope(ttn_ctx* c, const char* name, double flops, double bytes) : ctx(c) {
  ctx->launches++;
  ctx->flops_total += flops;
  if (ctx->launch_log && !ctx->capturing)
    std::fprintf(ctx->launch_log, "%s\t%.17g\t%.17g\n", name, flops, bytes);
  if (!ctx->profiling || ctx->capturing) return;
  int id = -1;
  for (size_t i = 0; i < ctx->prof_names.size(); ++i)
    if (ctx->prof_names[i] == name) id = (int)i;
  if (id < 0) {
    id = (int)ctx->prof_names.size();
    ctx->prof_names.push_back(name);
  }
  LaunchRecord r{id, pool_event(ctx), pool_event(ctx), flops, bytes};
  CUDA_CHECK(cudaEventRecord(r.start, ctx->stream));
  idx = (int)ctx->prof.size();
  ctx->prof.push_back(r);
}

LaunchScope::~LaunchScope() {
  if (idx >= 0) cudaEventRecord(ctx->prof[idx].stop, ctx->stream);
}

PhaseScope::PhaseScope(ttn_ctx* c, const char* name) : ctx(c) {
  if (!ctx->profiling || ctx->capturing) return;
  const std::string full = std::string("phase:") + name;
  int id = -1;
  for (size_t i = 0; i < ctx->prof_names.size(); ++i)
    if (ctx->prof_names[i] == full) id = (int)i;
  if (id < 0) {
    id = (int)ctx->prof_names.size();
    ctx->prof_names.push_back(full);
  }
  LaunchRecord r{id, pool_event(ctx), pool_event(ctx), 0.0, 0.0};
  CUDA_CHECK(cudaEventRecord(r.start, ctx->stream));
  idx = (int)ctx->prof.size();
  ctx->prof.push_back(r);
}

PhaseScope::~PhaseScope() {
  if (idx >= 0) cudaEventRecord(ctx->prof[idx].stop, ctx->stream);
}

template <class T>
void launch_gemm(ttn_ctx* ctx, const GemmDesc& g) {
  if (g.n_pairs <= 0 || g.st.n_sub <= 0 || g.M <= 0 || g.N <= 0) return;
  check_bounds(g, sizeof(T));
  long long nseg = 0;
  for (int s = 0; s < g.st.n_sub; ++s) nseg += g.hst->seg_ptr[s + 1] - g.hst->seg_ptr[s];
  int best = 0;
  long long best_cost = -1;
  for (int c = 0; c < 6; ++c) {
    const long long tm = (g.M + kCfgs[c].bm - 1) / kCfgs[c].bm;
    const long long tn = (g.N + kCfgs[c].bn - 1) / kCfgs[c].bn;
    const long long cost = tm * kCfgs[c].bm * tn * kCfgs[c].bn + tm * tn * 1024;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  const int tm = (g.M + kCfgs[best].bm - 1) / kCfgs[best].bm;
  const int tn = (g.N + kCfgs[best].bn - 1) / kCfgs[best].bn;
  const long long grid = (long long)tm * tn * g.st.n_sub * g.n_pairs;
  if (grid > 0x7fffffffLL) TTN_FAIL(TTN_EUNSUPPORTED, "gemm grid too large (%lld)", grid);
  static const char* names64[] = {"gemm_f64_64x64", "gemm_f64_64x32", "gemm_f64_32x32",
                                  "gemm_f64_128x16", "gemm_f64_64x16", "gemm_f64_16x16"};
  static const char* names32[] = {"gemm_f32_64x64", "gemm_f32_64x32", "gemm_f32_32x32",
                                  "gemm_f32_128x16", "gemm_f32_64x16", "gemm_f32_16x16"};
  const double flops = 2.0 * g.M * g.N * (double)g.K * nseg * g.n_pairs;
  const double bytes = algorithmic_bytes(g, sizeof(T));
  LaunchScope ls(ctx, sizeof(T) == 8 ? names64[best] : names32[best], flops, bytes);
  dispatch<T>(best, g, tm, tn, grid, ctx->stream);
  CUDA_LAUNCH_CHECK();
}

template <class T>
void launch_permute(ttn_ctx* ctx, const T* in, T* out, long long batch, int nd, const int* dims,
                    const int* perm) {
  PermArgs a{};
  a.nd = nd;
  long long stride[8], size = 1;
  for (int k = nd - 1; k >= 0; --k) {
    stride[k] = size;
    size *= dims[k];
  }
  for (int k = 0; k < nd; ++k) {
    a.od[k] = dims[perm[k]];
    a.is[k] = stride[perm[k]];
  }
  if (batch * size == 0) return;
  LaunchScope ls(ctx, "permute", 0.0, 1.0 * sizeof(T) * batch * size);   // node tensors read
  permute_kernel<T><<<grid_for(batch * size), kThreads, 0, ctx->stream>>>(in, out, batch, size,
                                                                          a);
  CUDA_LAUNCH_CHECK();
}

template <class T>
void launch_pair_dot(ttn_ctx* ctx, const T* bra, long long bra_stride, const T* Z,
                     long long z_stride, long long n, int n_pairs, const int* pair_bra,
                     double* out, int max_bra, long long bra_len, long long z_len) {
  if (n_pairs <= 0) return;
  TTN_REQUIRE((long long)max_bra * bra_stride + n <= bra_len &&
                  (long long)(n_pairs - 1) * z_stride + n <= z_len,
              "pair_dot bounds: bra %lld/%lld, Z %lld/%lld", (long long)max_bra * bra_stride + n,
              bra_len, (long long)(n_pairs - 1) * z_stride + n, z_len);
  LaunchScope ls(ctx, "pair_dot", 2.0 * n * n_pairs,
                 (double)sizeof(T) * n * std::min(n_pairs, max_bra + 1) + 8.0 * n_pairs);
  pair_dot_kernel<T><<<n_pairs, kThreads, 0, ctx->stream>>>(bra, bra_stride, Z, z_stride, n,
                                                             pair_bra, out);
  CUDA_LAUNCH_CHECK();
}

template <class T>
void launch_shift_axpy(ttn_ctx* ctx, T* y, const T* x, const double* shift, int n_states,
                       long long size) {
  const long long total = (long long)n_states * size;
  if (total == 0) return;
  LaunchScope ls(ctx, "shift_axpy", 2.0 * total, 3.0 * sizeof(T) * total);
  shift_axpy_kernel<T><<<grid_for(total), kThreads, 0, ctx->stream>>>(y, x, shift, size, total);
  CUDA_LAUNCH_CHECK();
}

void launch_to_f32(ttn_ctx* ctx, const double* in, float* out, long long n) {
  if (n == 0) return;
  LaunchScope ls(ctx, "to_f32", 0.0, 12.0 * n);
  to_f32_kernel<<<grid_for(n), kThreads, 0, ctx->stream>>>(in, out, n);
  CUDA_LAUNCH_CHECK();
}

void launch_to_f64(ttn_ctx* ctx, const float* in, double* out, long long n) {
  if (n == 0) return;
  LaunchScope ls(ctx, "to_f64", 0.0, 12.0 * n);
  to_f64_kernel<<<grid_for(n), kThreads, 0, ctx->stream>>>(in, out, n);
  CUDA_LAUNCH_CHECK();
}

void launch_gather_rows(ttn_ctx* ctx, double* dst, const double* src, const int* d_idx,
                        int n_rows, long long size) {
  const long long total = (long long)n_rows * size;
  if (total == 0) return;
  LaunchScope ls(ctx, "gather_states", 0.0, 16.0 * total);
  gather_rows_kernel<<<grid_for(total), kThreads, 0, ctx->stream>>>(dst, src, d_idx, size, total);
  CUDA_LAUNCH_CHECK();
}

void launch_count_nonfinite(ttn_ctx* ctx, const double* a, int rows, int cols, int ld,
                            unsigned* d_count) {
  CUDA_CHECK(cudaMemsetAsync(d_count, 0, sizeof(unsigned), ctx->stream));
  if ((long long)rows * cols == 0) return;
  LaunchScope ls(ctx, "count_nonfinite", 0.0, 8.0 * rows * cols);
  count_nonfinite_kernel<<<grid_for((long long)rows * cols), kThreads, 0, ctx->stream>>>(
      a, rows, cols, ld, d_count);
  CUDA_LAUNCH_CHECK();
}

void launch_scatter_gram(ttn_ctx* ctx, const double* g, int n_pairs, const int* pb,
                         const int* pk, int symmetric, double* out, int ld) {
  if (n_pairs <= 0) return;
  LaunchScope ls(ctx, "scatter_gram", 0.0, 24.0 * n_pairs);
  scatter_gram_kernel<<<(n_pairs + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
      g, n_pairs, pb, pk, symmetric, out, ld);
  CUDA_LAUNCH_CHECK();
}

// Groups per shared-memory chunk of the operator stage: up to 32 KB of d x d operators, at most
// 512 groups (their prefix indices are staged too).
template <class T, int D>
__host__ __device__ constexpr int op_stage_chunk() {
  constexpr int e = 8192 / (int)sizeof(T) * 4 / (D * D);
  return e < 1 ? 1 : (e > 512 ? 512 : e);
}

// One thread per output row r of one (pair, slot); all d outputs of the row in registers.
// The combined operators of the slot's groups are staged through shared memory in chunks;
// the output tile is transposed through shared memory so the global stores are coalesced.
template <class T, int D>
__global__ void __launch_bounds__(kThreads) op_stage_kernel(OpStageDesc o, int rtiles) {
  extern __shared__ unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  constexpr int GCH = op_stage_chunk<T, D>();
  T* sop = sh;
  T* sout = sh + GCH * D * D;                        // kThreads x (D + 1)
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int slot = (int)(rest % o.n_slots);
  const int pair = (int)(rest / o.n_slots);
  long long aidx = 0;
  if (o.A.mode == MODE_PAIR) aidx = pair;
  else if (o.A.mode == MODE_KET) aidx = o.pair_ket[pair];
  else if (o.A.mode == MODE_BRA) aidx = o.pair_bra[pair];
  const T* Tb = static_cast<const T*>(o.A.base) + aidx * o.A.pstride;
  const T* ops = static_cast<const T*>(o.ops);
  const int r0 = rt * (int)blockDim.x;   // row tile = blockDim.x rows (<= kThreads)
  const int r = r0 + threadIdx.x;
  T acc[D];
#pragma unroll
  for (int p = 0; p < D; ++p) acc[p] = T(0);
  const int g0 = o.slot_ptr[slot], g1 = o.slot_ptr[slot + 1];
  __shared__ int spre[GCH];
  for (int gc = g0; gc < g1; gc += GCH) {
    const int ng = min(GCH, g1 - gc);
    for (int i = threadIdx.x; i < ng * D * D; i += blockDim.x)
      sop[i] = ops[(long long)gc * D * D + i];
    for (int i = threadIdx.x; i < ng; i += blockDim.x) spre[i] = o.grp_prefix[gc + i];
    __syncthreads();
    if (r < o.rows) {
      int g = 0;
      // two groups at a time for small d (independent loads in flight); large d would spill
      for (; D <= 16 && g + 2 <= ng; g += 2) {
        const T* s0 = Tb + (long long)spre[g] * o.tsize + r;
        const T* s1 = Tb + (long long)spre[g + 1] * o.tsize + r;
        T t0[D], t1[D];
#pragma unroll
        for (int q = 0; q < D; ++q) {
          t0[q] = s0[(long long)q * o.rows];
          t1[q] = s1[(long long)q * o.rows];
        }
        const T* O0 = sop + g * D * D;
        const T* O1 = O0 + D * D;
#pragma unroll
        for (int q = 0; q < D; ++q)
#pragma unroll
          for (int p = 0; p < D; ++p)
            acc[p] = fma(O1[p * D + q], t1[q], fma(O0[p * D + q], t0[q], acc[p]));
      }
      for (; g < ng; ++g) {
        const T* src = Tb + (long long)spre[g] * o.tsize + r;
        const T* O = sop + g * D * D;
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const T t = src[(long long)q * o.rows];
#pragma unroll
          for (int p = 0; p < D; ++p) acc[p] = fma(O[p * D + q], t, acc[p]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < D; ++p) sout[threadIdx.x * (D + 1) + p] = acc[p];
  __syncthreads();
  T* Zb = static_cast<T*>(o.Z) + (long long)pair * o.z_pstride +
          (long long)slot * o.rows * D + (long long)r0 * D;
  const int nrow = min((int)blockDim.x, o.rows - r0);
  for (int i = threadIdx.x; i < nrow * D; i += blockDim.x)
    Zb[i] = sout[(i / D) * (D + 1) + (i % D)];
}

template <class T, int D>
static void op_stage_dispatch(ttn_ctx* ctx, const OpStageDesc& o, int rtiles, long long grid,
                              int tile) {
  constexpr int GCH = op_stage_chunk<T, D>();
  const size_t shmem = sizeof(T) * ((size_t)GCH * D * D + (size_t)kThreads * (D + 1));
  static int set_for_device[64] = {0};
  if (ctx->device >= 0 && ctx->device < 64 && !set_for_device[ctx->device]) {
    CUDA_CHECK(cudaFuncSetAttribute(op_stage_kernel<T, D>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem));
    set_for_device[ctx->device] = 1;
  }
  op_stage_kernel<T, D><<<grid, tile, shmem, ctx->stream>>>(o, rtiles);
}

template <class T>
void launch_op_stage(ttn_ctx* ctx, const OpStageDesc& o) {
  if (o.n_pairs <= 0 || o.n_slots <= 0 || o.rows <= 0) return;
  TTN_REQUIRE(o.d >= 1 && o.d <= 32, "operator stage: d = %d unsupported", o.d);
  long long base_max = 0;
  if (o.A.mode == MODE_PAIR) base_max = (long long)(o.n_pairs - 1) * o.A.pstride;
  else if (o.A.mode == MODE_KET) base_max = (long long)o.max_ket * o.A.pstride;
  TTN_REQUIRE(o.n_groups == 0 || base_max + (long long)(o.max_prefix + 1) * o.tsize <= o.a_len,
              "op stage bounds: A reaches %lld of %lld",
              base_max + (long long)(o.max_prefix + 1) * o.tsize, o.a_len);
  TTN_REQUIRE((long long)o.n_pairs * o.z_pstride <= o.z_len &&
                  (long long)o.n_slots * o.rows * o.d <= o.z_pstride,
              "op stage bounds: Z");
  // row tiles split the rows evenly, in whole warps (576 rows: 3 x 192; 9 rows: 1 x 32)
  const int nt = (o.rows + kThreads - 1) / kThreads;
  const int tile = ((o.rows + nt - 1) / nt + 31) / 32 * 32;
  const int rtiles = (o.rows + tile - 1) / tile;
  const long long grid = (long long)rtiles * o.n_slots * o.n_pairs;
  TTN_REQUIRE(grid <= 0x7fffffffLL, "op stage grid too large");
  const double flops = 2.0 * o.d * o.d * (double)o.rows * o.n_groups * o.n_pairs;
  const double in_bases = o.A.mode == MODE_KET ? std::min(o.n_pairs, o.max_ket + 1) : o.n_pairs;
  const double bytes =
      (double)sizeof(T) * ((o.alg_in ? in_bases * o.n_unique_prefix * o.tsize : 0.0) +
                           (o.alg_out ? (double)o.n_pairs * o.n_slots * o.rows * o.d : 0.0));
  LaunchScope ls(ctx, sizeof(T) == 8 ? "op_stage_f64" : "op_stage_f32", flops, bytes);
  switch (o.d) {
#define TTN_OPD(k) case k: op_stage_dispatch<T, k>(ctx, o, rtiles, grid, tile); break;
    TTN_OPD(1) TTN_OPD(2) TTN_OPD(3) TTN_OPD(4) TTN_OPD(5) TTN_OPD(6) TTN_OPD(7) TTN_OPD(8)
    TTN_OPD(9) TTN_OPD(10) TTN_OPD(11) TTN_OPD(12) TTN_OPD(13) TTN_OPD(14) TTN_OPD(15)
    TTN_OPD(16) TTN_OPD(17) TTN_OPD(18) TTN_OPD(19) TTN_OPD(20) TTN_OPD(21) TTN_OPD(22)
    TTN_OPD(23) TTN_OPD(24) TTN_OPD(25) TTN_OPD(26) TTN_OPD(27) TTN_OPD(28) TTN_OPD(29)
    TTN_OPD(30) TTN_OPD(31) TTN_OPD(32)
#undef TTN_OPD
  }
  CUDA_LAUNCH_CHECK();
}

// Level stage of a node contraction, specialised for its shape: out[r][a] = sum_b in[b][r] E[a][b]
// with rows r up to ~1e4 and a, b <= 64. One thread per row keeps all NA outputs in registers;
// the environment slice is staged transposed (Es[b][a], zero-padded to NA) in shared memory and
// read with broadcast vector loads; each item has exactly one segment.
template <class T, int NA>
__global__ void __launch_bounds__(kThreads) level_kernel(GemmDesc g, int rtiles) {
  constexpr int KMAX = 64;
  // the output tile (kThreads rows x NA, rows contiguous in global memory) is staged through a
  // padded shared buffer so the global stores are coalesced; only where it fits statically
  constexpr bool kStage = sizeof(T) == 4 && NA <= 32;
  constexpr int kOutLd = NA + 1;
  __shared__ __align__(16) T Es[KMAX * NA];
  __shared__ T Os[kStage ? kThreads * kOutLd : 1];
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int sub = (int)(rest % g.st.n_sub);
  const int pair = (int)(rest / g.st.n_sub);
  const T* Abase = operand_base<T>(g.A, pair, g.pair_bra, g.pair_ket);
  const T* Bbase = operand_base<T>(g.B, pair, g.pair_bra, g.pair_ket);
  const int r0 = rt * kThreads;
  const int r = r0 + threadIdx.x;
  const bool live = r < g.M;
  T acc[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) acc[a] = T(0);
  for (int seg = g.st.seg_ptr[sub]; seg < g.st.seg_ptr[sub + 1]; ++seg) {
  const T* Ab = Abase + g.st.seg_a[seg];
  const T* Bb = Bbase + g.st.seg_b[seg];
  __syncthreads();
  for (int i = threadIdx.x; i < g.K * NA; i += kThreads) {
    const int b = i / NA, a = i % NA;
    Es[i] = a < g.N ? Bb[(long long)a * g.b_sn + (long long)b * g.b_sk] : T(0);
  }
  __syncthreads();
  if (live) {
    const T* src = Ab + r;
    int b = 0;
    for (; b + 8 <= g.K; b += 8) {
      T t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = src[(long long)(b + u) * g.a_sk];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T* e = Es + (b + u) * NA;
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = fma(e[a], t[u], acc[a]);
      }
    }
    for (; b < g.K; ++b) {
      const T t = src[(long long)b * g.a_sk];
      const T* e = Es + b * NA;
#pragma unroll
      for (int a = 0; a < NA; ++a) acc[a] = fma(e[a], t, acc[a]);
    }
  }
  }
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  T* base = static_cast<T*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub];
  if constexpr (kStage) {
#pragma unroll
    for (int a = 0; a < NA; ++a) Os[threadIdx.x * kOutLd + a] = acc[a];
    __syncthreads();
    const int nrow = min(kThreads, g.M - r0);
    T* dst = base + (long long)r0 * g.c_sm;     // c_sm == N: the tile is contiguous
    for (int i = threadIdx.x; i < nrow * g.N; i += kThreads)
      dst[i] = Os[(i / g.N) * kOutLd + (i % g.N)];
  } else {
    if (!live) return;
    T* dst = base + (long long)r * g.c_sm;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (a < g.N) dst[a] = acc[a];
  }
}

// True if the descriptor has the level-stage shape the specialised kernel handles.
bool level_shape_ok(const GemmDesc& g) {
  return g.a_sm == 1 && g.c_sn == 1 && g.c_sm == g.N && g.K <= 64 && g.N <= 64;
}

// Et[pair][G] = sum_{t in G} coef_t E[pair][w_t], written transposed: E slices are [a][b]
// (da x db), Et slices [b][a], so the segmented level stage that consumes Et can take each
// slice into shared memory as it lands (the layout its thread tiles read).
template <class T>
__global__ void combine_env_kernel(const T* __restrict__ E, long long e_pstride, int da, int db,
                                   T* __restrict__ Et, int nG, const int* __restrict__ term_ptr,
                                   const int* __restrict__ term_w,
                                   const T* __restrict__ term_coef, long long total) {
  const long long eslice = (long long)da * db;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long per_pair = (long long)nG * eslice;
    const long long pair = idx / per_pair;
    const long long r = idx - pair * per_pair;
    const int G = (int)(r / eslice);
    const int e_t = (int)(r - (long long)G * eslice);   // b * da + a
    const int b = e_t / da, a = e_t - b * da;
    const T* Ep = E + pair * e_pstride + (long long)a * db + b;
    T acc = T(0);
    for (int t = term_ptr[G]; t < term_ptr[G + 1]; ++t)
      acc = fma(term_coef[t], Ep[(long long)term_w[t] * eslice], acc);
    Et[idx] = acc;
  }
}

template <class T>
void launch_combine_env(ttn_ctx* ctx, const T* E, long long e_pstride, int da, int db, T* Et,
                        int n_pairs, int nG, const int* term_ptr, const int* term_w,
                        const T* term_coef, int max_w) {
  const long long eslice = (long long)da * db;
  const long long total = (long long)n_pairs * nG * eslice;
  if (total == 0) return;
  TTN_REQUIRE((long long)(max_w + 1) * eslice <= e_pstride, "combine bounds");
  // algorithmic bytes: the distinct environment slices read (Et is an intermediate)
  LaunchScope ls(ctx, sizeof(T) == 8 ? "combine_env_f64" : "combine_env_f32", 2.0 * total,
                 (double)sizeof(T) * n_pairs * (max_w + 1) * eslice);
  long long blocks = (total + kThreads - 1) / kThreads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  combine_env_kernel<T><<<(int)blocks, kThreads, 0, ctx->stream>>>(E, e_pstride, da, db, Et, nG,
                                                                 term_ptr, term_w, term_coef,
                                                                 total);
  CUDA_LAUNCH_CHECK();
}

template void launch_combine_env<double>(ttn_ctx*, const double*, long long, int, int, double*,
                                         int, int, const int*, const int*, const double*, int);
template void launch_combine_env<float>(ttn_ctx*, const float*, long long, int, int, float*,
                                        int, int, const int*, const int*, const float*, int);

// ---- bulk copies (cp.async.bulk, the 1-D TMA path) completing on an mbarrier --------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// global -> shared tensor copy of one box at element coordinates (x, y) of a 2-D tensor map
// (x * 4 bytes a multiple of 16; the destination 128-byte aligned); elements outside the tensor
// land as zeros and count towards the barrier's bytes like the others
__device__ __forceinline__ void tensor_copy_g2s(void* dst, const CUtensorMap* map, int x, int y,
                                                unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
      "[%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
// Orders earlier generic-proxy accesses of shared memory before later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for phase `parity` of the barrier; gives up after budget_ns of device time (2 s for
// the bulk-copy kernels), writes flag_value into the context's wait flag and returns false (the
// caller then leaves the CTA without touching the staged data). A wait that has already lasted
// 1 ms also gives up, without writing, once another CTA has set the flag, so that a launch whose
// waits cannot complete ends after one budget instead of one budget per CTA.
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;
constexpr unsigned long long kWaitPeerCheckNs = 1000000ull;
// second, short wait for work still in flight after a wait gave up
constexpr unsigned long long kWaitDrainNs = 10000000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned* flag,
                                          unsigned long long budget_ns = kWaitBudgetNs,
                                          unsigned flag_value = TTN_WAIT_FLAG_COPY) {
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 255u) {
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (flag && now - t0 > kWaitPeerCheckNs &&
                 *reinterpret_cast<volatile unsigned*>(flag) != 0u) {
        return false;
      } else if (now - t0 > budget_ns) {
        if (flag) {
          *reinterpret_cast<volatile unsigned*>(flag) = flag_value;
          __threadfence_system();
        }
        return false;
      }
    }
  }
}

// ---- level stage on bulk-copied tiles (float32 data) --------------------------------------------
// out[r][a] = sum_b A[b][r] E[a][b] with the A tile (K rows of rows_cta contiguous floats, row
// stride lda) and the environment slices E[a][b] (N x K contiguous) brought to shared memory by
// bulk copies. A warp owns 32 rows of the tile and all NA (>= N, a multiple of 8) columns.
//  * SIMT (TC = false): each thread owns 4 consecutive rows x NA/4 columns; the slice is
//    transposed once to Es[b][a]; per b one 16-byte load of A, NA/8 8-byte loads of Es and
//    4 * NA/4 FMAs. lda = rows_cta.
//  * Tensor cores (TC = true, the TTN_TF32X3 precision): the warp's rows are two 16-row MMA
//    tiles; mma.sync m16n8k8 TF32 with the 3xTF32 split x = hi + lo, hi = tf32(x),
//    lo = tf32(x - hi), each product formed as lo*hi + hi*lo + hi*hi with float32 accumulation
//    (relative error of a product ~2^-21 instead of ~2^-11 for plain TF32). The slice is split
//    once into Eh/El[n][k] (row stride K + 4: conflict-free B fragments); A fragments are split
//    on the fly. lda = rows_cta + 8 (conflict-free A fragments). Needs K % 8 == 0.
// Fragment layout of m16n8k8 .row.col: groupID gq = lane / 4, tq = lane % 4; A: (gq, tq),
// (gq + 8, tq), (gq, tq + 4), (gq + 8, tq + 4); B: (k = tq, n = gq), (k = tq + 4, n = gq);
// C: (gq, 2tq), (gq, 2tq + 1), (gq + 8, 2tq), (gq + 8, 2tq + 1).
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_m16n8k8_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// floats of one staged environment slice in the compute layout
template <int NA, bool TC>
__host__ __device__ __forceinline__ int level_env_floats(int K) {
  return TC ? 2 * NA * (K + 4) : K * NA;
}

// raw slice (Er[a * K + b], or Er[b * N + a] when et) -> compute layout (padding columns zero);
// whole CTA
template <int NA, bool TC>
__device__ __forceinline__ void level_stage_env(const float* Er, float* Ec, int N, int K, bool et) {
  if constexpr (TC) {
    uint32_t* Eh = reinterpret_cast<uint32_t*>(Ec);
    uint32_t* El = Eh + NA * (K + 4);
    for (int i = threadIdx.x; i < NA * K; i += blockDim.x) {
      const int n = i / K, k = i - n * K;
      const float x = n < N ? Er[et ? k * N + n : n * K + k] : 0.f;
      const uint32_t hi = tf32_bits(x);
      Eh[n * (K + 4) + k] = hi;
      El[n * (K + 4) + k] = tf32_bits(x - __uint_as_float(hi));
    }
  } else {
    for (int i = threadIdx.x; i < K * NA; i += blockDim.x) {
      const int b = i / NA, a = i - b * NA;
      Ec[i] = a < N ? Er[et ? b * N + a : a * K + b] : 0.f;
    }
  }
}

// acc (NA floats per thread) += this warp's 32 rows of A x the staged slice
template <int NA, bool TC>
__device__ __forceinline__ void level_mac(const float* As, int lda, const float* Ec, int K,
                                          float* acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (TC) {
    constexpr int NT = NA / 8;
    const uint32_t* Eh = reinterpret_cast<const uint32_t*>(Ec);
    const uint32_t* El = Eh + NA * (K + 4);
    const int gq = lane >> 2, tq = lane & 3, rw = warp * 32;
    for (int k0 = 0; k0 < K; k0 += 8) {
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const float* ap = As + (k0 + tq) * lda + rw + m * 16 + gq;
        const float x[4] = {ap[0], ap[8], ap[4 * lda], ap[4 * lda + 8]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ah[m][q] = tf32_bits(x[q]);
          al[m][q] = tf32_bits(x[q] - __uint_as_float(ah[m][q]));
        }
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int off = (j * 8 + gq) * (K + 4) + k0 + tq;
        const uint32_t bh[2] = {Eh[off], Eh[off + 4]};
        const uint32_t bl[2] = {El[off], El[off + 4]};
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          float* d = acc + (m * NT + j) * 4;
          mma_m16n8k8_tf32(d, al[m], bh);
          mma_m16n8k8_tf32(d, ah[m], bl);
          mma_m16n8k8_tf32(d, ah[m], bh);
        }
      }
    }
  } else {
    constexpr int CPT = NA / 4;
    const int rl = warp * 32 + (lane >> 2) * 4, cg = lane & 3;
    const float* es = Ec + cg * CPT;
#pragma unroll 4
    for (int b = 0; b < K; ++b) {
      const float4 x4 = *reinterpret_cast<const float4*>(As + b * lda + rl);
      const float x[4] = {x4.x, x4.y, x4.z, x4.w};
      float e[CPT];
#pragma unroll
      for (int c = 0; c < CPT; c += 2) {
        const float2 v = *reinterpret_cast<const float2*>(es + b * NA + c);
        e[c] = v.x;
        e[c + 1] = v.y;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[i * CPT + c] = fmaf(x[i], e[c], acc[i * CPT + c]);
    }
  }
}

// rows [0, nrow) of the tile whose first row is at dst (row stride N)
template <int NA, bool TC>
__device__ __forceinline__ void level_store(float* dst, int nrow, int N, const float* acc,
                                            int vec_store) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (TC) {
    constexpr int NT = NA / 8;
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = warp * 32 + m * 16 + gq + 8 * h;
        if (r >= nrow) continue;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const int col = j * 8 + 2 * tq;
          const float* v = acc + (m * NT + j) * 4 + 2 * h;
          float* o = dst + (long long)r * N + col;
          if (vec_store) {
            *reinterpret_cast<float2*>(o) = make_float2(v[0], v[1]);
          } else {
            if (col < N) o[0] = v[0];
            if (col + 1 < N) o[1] = v[1];
          }
        }
      }
  } else {
    constexpr int CPT = NA / 4;
    const int rl = warp * 32 + (lane >> 2) * 4, cg = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (rl + i >= nrow) break;
      float* o = dst + (long long)(rl + i) * N + cg * CPT;
      if (vec_store) {
#pragma unroll
        for (int c = 0; c < CPT; c += 2)
          *reinterpret_cast<float2*>(o + c) = make_float2(acc[i * CPT + c], acc[i * CPT + c + 1]);
      } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c)
          if (cg * CPT + c < N) o[c] = acc[i * CPT + c];
      }
    }
  }
}

// One CTA takes one row tile of one A group, i.e. up to sb_max single-segment items of one
// pair that read the same A slice: the A tile and every item's slice land on one mbarrier, each
// slice is brought to the compute layout, and the items are computed one after the other from
// the one staged tile.
template <int NA, bool TC, bool TMAP>
__global__ void __launch_bounds__(288) level_tma_kernel(GemmDesc g, int rtiles, int rows_cta,
                                                        int sb_max, int vec_store, int et,
                                                        const __grid_constant__ CUtensorMap tmA) {
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) unsigned long long bar;
  const int lda = TC ? rows_cta + 8 : rows_cta;
  const int nk4 = (g.N * g.K + 3) & ~3;
  const int esz = level_env_floats<NA, TC>(g.K);
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int q = (int)(rest % g.st.n_grp);
  const int pair = (int)(rest / g.st.n_grp);
  const int gs = g.st.grp_ptr[q], ns = g.st.grp_ptr[q + 1] - gs;
  const int r0 = rt * rows_cta;
  const int nrow = min(rows_cta, g.M - r0);
  const float* Abase = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket);
  const float* Bbase = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket);
  float* As = dsm;
  float* Er = dsm + g.K * lda;
  float* Ec = Er + sb_max * nk4;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float* Ab = Abase + g.st.grp_a[q] + r0;
    if (TMAP && (smem_addr(dsm) & 127u) == 0u) {
      // the A tile as one tensor copy (a box of lda x K of the buffer's row view)
      const long long oa = Abase + g.st.grp_a[q] - static_cast<const float*>(g.A.base);
      mbar_expect_tx(&bar, (unsigned)(g.K * lda + ns * g.N * g.K) * 4u);
      tensor_copy_g2s(As, &tmA, r0, (int)(oa / g.a_sk), &bar);
    } else {
      mbar_expect_tx(&bar, (unsigned)(g.K * nrow + ns * g.N * g.K) * 4u);
      for (int b = 0; b < g.K; ++b)
        bulk_copy_g2s(As + b * lda, Ab + (long long)b * g.a_sk, nrow * 4u, &bar);
    }
    for (int j = 0; j < ns; ++j)
      bulk_copy_g2s(Er + j * nk4, Bbase + g.st.grp_b[gs + j], g.N * g.K * 4u, &bar);
  }
  const bool ok = mbar_wait(&bar, 0, g.wait_flag);
  if (__syncthreads_or(!ok)) return;
  for (int j = 0; j < ns; ++j)
    level_stage_env<NA, TC>(Er + j * nk4, Ec + j * esz, g.N, g.K, et != 0);
  __syncthreads();
  if ((threadIdx.x >> 5) * 32 >= nrow) return;   // whole warps only (MMA needs all lanes)
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  float* Cpair = static_cast<float*>(g.C) + cidx * g.c_pstride;
  for (int j = 0; j < ns; ++j) {
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.f;
    level_mac<NA, TC>(As, lda, Ec + j * esz, g.K, acc);
    level_store<NA, TC>(Cpair + g.st.grp_c[gs + j] + (long long)r0 * g.N, nrow, g.N, acc,
                        vec_store);
  }
}

// Items that sum several segments (the segmented last level of the operator-first order):
// Z[item] = sum_seg A_seg x E_seg. One CTA takes one row tile of one item; each segment's A tile
// and slice land in one stage of a two-stage ring of mbarrier-tracked bulk copies (segment j + 2
// is requested once segment j has been consumed) and accumulate in registers.
template <int NA, bool TC>
__global__ void __launch_bounds__(288) level_tma_seg_kernel(GemmDesc g, int rtiles, int rows_cta,
                                                            int vec_store, int et) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ __align__(8) unsigned long long bar[2];
  const int lda = TC ? rows_cta + 8 : rows_cta;
  const int nk4 = (g.N * g.K + 3) & ~3;
  const int stage = g.K * lda + nk4 + level_env_floats<NA, TC>(g.K);
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int sub = (int)(rest % g.st.n_sub);
  const int pair = (int)(rest / g.st.n_sub);
  const int s0 = g.st.seg_ptr[sub], nseg = g.st.seg_ptr[sub + 1] - s0;
  const int r0 = rt * rows_cta;
  const int nrow = min(rows_cta, g.M - r0);
  const float* Abase = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket);
  const float* Bbase = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket);
  auto issue = [&](int j, int st) {
    float* As = dsm + st * stage;
    float* Er = As + g.K * lda;
    const float* Ab = Abase + g.st.seg_a[s0 + j] + r0;
    mbar_expect_tx(&bar[st], (unsigned)(g.K * nrow + g.N * g.K) * 4u);
    for (int b = 0; b < g.K; ++b)
      bulk_copy_g2s(As + b * lda, Ab + (long long)b * g.a_sk, nrow * 4u, &bar[st]);
    bulk_copy_g2s(Er, Bbase + g.st.seg_b[s0 + j], g.N * g.K * 4u, &bar[st]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (nseg > 0) issue(0, 0);
    if (nseg > 1) issue(1, 1);
  }
  const bool live = (threadIdx.x >> 5) * 32 < nrow;   // warp-uniform
  float acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = 0.f;
  unsigned phase[2] = {0u, 0u};
  for (int j = 0; j < nseg; ++j) {
    const int st = j & 1;
    const bool ok = mbar_wait(&bar[st], phase[st], g.wait_flag);
    phase[st] ^= 1u;
    if (__syncthreads_or(!ok)) return;
    const float* As = dsm + st * stage;
    const float* Er = As + g.K * lda;
    float* Ec = const_cast<float*>(Er) + nk4;
    level_stage_env<NA, TC>(Er, Ec, g.N, g.K, et != 0);
    __syncthreads();
    if (live) level_mac<NA, TC>(As, lda, Ec, g.K, acc);
    __syncthreads();
    if (threadIdx.x == 0 && j + 2 < nseg) {
      fence_proxy_async();
      issue(j + 2, st);
    }
  }
  if (!live) return;
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  level_store<NA, TC>(static_cast<float*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub] +
                          (long long)r0 * g.N,
                      nrow, g.N, acc, vec_store);
}


__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Self-test of the bounded wait: one thread arrives on the barrier announcing 16 bytes of
// transfer that no copy will ever deliver, so the phase cannot complete; every thread then
// waits with the given budget, which runs out. No copy is in flight when the CTA leaves.
__global__ void wait_selftest_kernel(unsigned* flag, unsigned long long budget_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, 16u);
  mbar_wait(&bar, 0, flag, budget_ns, TTN_WAIT_FLAG_SELFTEST);
}

void launch_wait_selftest(ttn_ctx* ctx, unsigned long long budget_ns) {
  LaunchScope ls(ctx, "wait_selftest", 0.0, 0.0);
  wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_wait, budget_ns);
  CUDA_LAUNCH_CHECK();
}

// acc += this warp's 32 rows of A (shared, K rows of lda floats) x a raw slice Er[k][n] (row
// length N = NA) on the tensor cores: mma.sync m16n8k8 TF32 with the 3xTF32 split of both
// operands, B fragments split as they are read (the raw [k][n] slice gives conflict-free
// fragment loads for N = 8, 16, 24, 32). lda = rows + 8 keeps the A fragment loads
// conflict-free. acc holds the m16n8 accumulator fragments (2 m tiles x NA/8 n tiles x 4).
template <int NA>
__device__ __forceinline__ void level_mac_raw_tc(const float* As, int lda, const float* Er, int K,
                                                 float* acc) {
  constexpr int NT = NA / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3, rw = warp * 32;
  for (int k0 = 0; k0 < K; k0 += 8) {
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const float* ap = As + (k0 + tq) * lda + rw + m * 16 + gq;
      const float x[4] = {ap[0], ap[8], ap[4 * lda], ap[4 * lda + 8]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[m][q] = tf32_bits(x[q]);
        al[m][q] = tf32_bits(x[q] - __uint_as_float(ah[m][q]));
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const float e0 = Er[(k0 + tq) * NA + j * 8 + gq];
      const float e1 = Er[(k0 + tq + 4) * NA + j * 8 + gq];
      uint32_t bh[2], bl[2];
      bh[0] = tf32_bits(e0);
      bl[0] = tf32_bits(e0 - __uint_as_float(bh[0]));
      bh[1] = tf32_bits(e1);
      bl[1] = tf32_bits(e1 - __uint_as_float(bh[1]));
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        float* d = acc + (m * NT + j) * 4;
        mma_m16n8k8_tf32(d, al[m], bh);
        mma_m16n8k8_tf32(d, ah[m], bl);
        mma_m16n8k8_tf32(d, ah[m], bh);
      }
    }
  }
}

// Floats of one stage of the warp-specialised segmented level kernel: the A tile (K rows of lda)
// and the slice (K x NA), rounded up to 128 bytes so that every stage starts 128-byte aligned.
__host__ __device__ inline int seg_ws_stage_floats(int K, int lda, int na) {
  return (K * lda + K * na + 31) & ~31;
}

// Segmented level stage, warp-specialised (slices stored [b][a] with N = NA, i.e. already in
// the SIMT compute layout). Warps 0..nw-1 compute (32 rows each; float32 SIMT, or the
// tensor-core 3xTF32 path when TC), warp nw produces: its first lane requests segment j's A
// tile and slice into stage j % 2 once the compute warps have released that stage (an "empty"
// mbarrier with one arrival per compute warp), and the copies complete a "full" mbarrier the
// compute warps wait on. No CTA-wide barrier inside the segment loop; every wait is bounded.
// A tile rows are lda = rows_cta (+ 8 for TC) floats apart.
// TMAP: the A tile comes as one tensor copy (a box of lda x K from the row view of the A
// buffer, rows a_sk floats long) instead of K row copies, where the destination is 128-byte
// aligned (the row copies stand in otherwise).
template <int NA, bool TC, bool TMAP>
__device__ __forceinline__ bool seg_ws_pipeline(const GemmDesc& g, float* dsm, int rows_cta,
                                                int lda, int stage, int pair, int s0, int nseg,
                                                int r0, int nrow, unsigned long long* full,
                                                unsigned long long* empty, float* acc,
                                                const CUtensorMap* tmA) {
  const int nw = rows_cta >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == nw) {
    if (lane == 0) {
      const float* Abase = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket);
      const float* Bbase = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket);
      for (int j = 0; j < nseg; ++j) {
        const int st = j & 1;
        if (j >= 2 && !mbar_wait(&empty[st], ((j >> 1) - 1) & 1, g.wait_flag)) break;
        fence_proxy_async();
        float* As = dsm + st * stage;
        float* Es = As + g.K * lda;
        const float* Ab = Abase + g.st.seg_a[s0 + j] + r0;
        if (TMAP && (smem_addr(dsm) & 127u) == 0u) {
          const long long oa = Abase + g.st.seg_a[s0 + j] - static_cast<const float*>(g.A.base);
          mbar_expect_tx(&full[st], (unsigned)(g.K * lda + g.N * g.K) * 4u);
          tensor_copy_g2s(As, tmA, r0, (int)(oa / g.a_sk), &full[st]);
        } else {
          mbar_expect_tx(&full[st], (unsigned)(g.K * nrow + g.N * g.K) * 4u);
          for (int b = 0; b < g.K; ++b)
            bulk_copy_g2s(As + b * lda, Ab + (long long)b * g.a_sk, nrow * 4u, &full[st]);
        }
        bulk_copy_g2s(Es, Bbase + g.st.seg_b[s0 + j], g.N * g.K * 4u, &full[st]);
      }
    }
    return false;
  }
  const bool live = warp * 32 < nrow;   // warp-uniform
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = 0.f;
  for (int j = 0; j < nseg; ++j) {
    const int st = j & 1;
    if (!mbar_wait(&full[st], (j >> 1) & 1, g.wait_flag)) return false;
    const float* As = dsm + st * stage;
    if (live) {
      if constexpr (TC) level_mac_raw_tc<NA>(As, lda, As + g.K * lda, g.K, acc);
      else level_mac<NA, false>(As, lda, As + g.K * lda, g.K, acc);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  return true;
}

template <int NA, bool TC, bool TMAP>
__global__ void __launch_bounds__(320) level_seg_ws_kernel(GemmDesc g, int rtiles, int rows_cta,
                                                           int vec_store,
                                                           const __grid_constant__ CUtensorMap tmA) {
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) unsigned long long full[2];
  __shared__ __align__(8) unsigned long long empty[2];
  const int nw = rows_cta >> 5;
  const int lda = rows_cta + (TC ? 8 : 0);
  const int stage = seg_ws_stage_floats(g.K, lda, NA);
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int sub = (int)(rest % g.st.n_sub);
  const int pair = (int)(rest / g.st.n_sub);
  const int s0 = g.st.seg_ptr[sub], nseg = g.st.seg_ptr[sub + 1] - s0;
  const int r0 = rt * rows_cta;
  const int nrow = min(rows_cta, g.M - r0);
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], nw);
    mbar_init(&empty[1], nw);
    mbar_init_fence();
  }
  __syncthreads();
  float acc[NA];
  if (!seg_ws_pipeline<NA, TC, TMAP>(g, dsm, rows_cta, lda, stage, pair, s0, nseg, r0, nrow,
                                     full, empty, acc, &tmA))
    return;
  if ((threadIdx.x >> 5) * 32 >= nrow) return;
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  level_store<NA, TC>(static_cast<float*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub] +
                          (long long)r0 * g.N,
                      nrow, g.N, acc, vec_store);
}

// ---- level stage on the fifth-generation tensor cores (tcgen05.mma, tensor-memory accumulators)
// The grouped level stage C_j[r][a] = sum_b A[b][r] E_j[a][b] of one A group (the items j that
// read the same A slice, i.e. the children of one prefix in the TTNO trie) for a 128-row tile:
//  * the A tile (K slices of up to 128 contiguous rows; one tensor-map box where the buffer has
//    a row view, else one bulk copy per slice) and the group's environment slices arrive on an
//    mbarrier, requested while the previous work item is finished;
//  * both operands are split x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) into the K-major,
//    non-swizzled layout the shared-memory matrix descriptors address: core matrices of 8 rows x
//    16 bytes, K-adjacent core matrices 128 bytes apart (leading byte offset), consecutive 8-row
//    groups 32 * Kp bytes apart (stride byte offset), Kp = K rounded up to 8 with zero padding;
//  * one thread issues tcgen05.mma kind::tf32 (M = 128, N = items x NA rounded up to 16, K = 8
//    per instruction), lo*hi + hi*lo + hi*hi per K step, float32 accumulation in tensor memory
//    (the 3xTF32 product, ~2^-21 relative per product); a group with more items than fit in
//    the CTA's accumulator columns (at most 128) runs in several passes;
//  * warp w reads tensor-memory lanes 32w..32w+31 (= rows) back with tcgen05.ld and writes them
//    through its staging tile with one bulk store.
// Every wait is bounded (2 s); after a timeout the CTA waits once more, then frees its tensor
// memory and leaves, and the host reports TTN_ETIMEOUT.
constexpr int kUmmaRows = 128;   // MMA M: one accumulator lane per row

// shared-memory matrix descriptor: start address, leading byte offset 128, stride byte offset,
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t umma_sdesc(unsigned addr, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(unsigned d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          int accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrives once on the barrier when every MMA this thread issued so far has completed
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared -> global bulk copy (both addresses 16-byte aligned, bytes a multiple of 16), tracked
// by this thread's bulk groups
__device__ __forceinline__ void bulk_store_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// waits until at most one of this thread's bulk stores still reads its shared-memory source
__device__ __forceinline__ void bulk_store_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_store_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// NA consecutive float32 columns of this thread's lane: the loads of one row and a single
// wait in one asm statement (the destination registers are not valid before the wait)
template <int NA>
__device__ __forceinline__ void tmem_ld_row(unsigned taddr, float* v) {
  uint32_t r[NA];
  if constexpr (NA == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
  } else if constexpr (NA == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
  } else if constexpr (NA == 24) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(taddr), "r"(taddr + 16u)
        : "memory");
  } else {
    static_assert(NA == 32, "row width");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
  }
#pragma unroll
  for (int i = 0; i < NA; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of one 128 x N tile, warp by warp (no CTA barrier): warp w's 32 rows (v = this
// thread's row) go to its own staging tile (two per warp, alternating) and out with one bulk
// store issued by the warp's first lane, or with direct stores when bulk_out is 0. `n_out`
// counts the warp's bulk stores (its first lane's bulk groups).
template <int NA>
__device__ __forceinline__ void umma_store_tile(float* o, int nrow, int N, const float* v,
                                                float* stage_warp, int& n_out, int bulk_out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nr = min(32, nrow - warp * 32);
  if (nr <= 0) return;
  float* ow = o + (long long)warp * 32 * N;
  if (bulk_out) {
    float* st = stage_warp + (n_out & 1) * 32 * N;
    if (lane == 0) bulk_store_wait_read1();   // the store that last read this tile is done
    __syncwarp();
    if (lane < nr) {
#pragma unroll
      for (int c = 0; c < NA; c += 4)
        if (c < N)
          *reinterpret_cast<float4*>(st + lane * N + c) =
              make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
    }
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) bulk_store_s2g(ow, st, (unsigned)(nr * N) * 4u);
    ++n_out;
  } else if (lane < nr) {
#pragma unroll
    for (int c = 0; c < NA; ++c)
      if (c < N) ow[(long long)lane * N + c] = v[c];
  }
}

// hi / lo parts of 4 K-consecutive values of row n into the canonical K-major layout
__device__ __forceinline__ void umma_store_split(uint32_t* hi, uint32_t* lo, int n, int kq, int kp,
                                                 const float* x) {
  const int off = (n & 7) * 4 + (n >> 3) * 8 * kp + kq * 32;
  uint4 h, l;
  h.x = tf32_bits(x[0]);
  h.y = tf32_bits(x[1]);
  h.z = tf32_bits(x[2]);
  h.w = tf32_bits(x[3]);
  l.x = tf32_bits(x[0] - __uint_as_float(h.x));
  l.y = tf32_bits(x[1] - __uint_as_float(h.y));
  l.z = tf32_bits(x[2] - __uint_as_float(h.z));
  l.w = tf32_bits(x[3] - __uint_as_float(h.w));
  *reinterpret_cast<uint4*>(hi + off) = h;
  *reinterpret_cast<uint4*>(lo + off) = l;
}

// Shared-memory plan of one CTA (byte offsets, each region 128-byte aligned).
struct UmmaLevelSmem {
  size_t raw_a, raw_e, a_hi, a_lo, b_hi, b_lo, stage, total;
};
__host__ __device__ inline size_t umma_align(size_t x) { return (x + 127) & ~(size_t)127; }
__host__ __device__ inline UmmaLevelSmem umma_level_plan(int K, int kp, int N, int sb_max,
                                                         int nb_rows) {
  UmmaLevelSmem p;
  const size_t nk4 = (size_t)((N * K + 3) & ~3);
  p.raw_a = 0;
  p.raw_e = umma_align(p.raw_a + 4 * (size_t)K * kUmmaRows);
  p.a_hi = umma_align(p.raw_e + 4 * (size_t)sb_max * nk4);
  p.a_lo = umma_align(p.a_hi + 4 * (size_t)kUmmaRows * kp);
  p.b_hi = umma_align(p.a_lo + 4 * (size_t)kUmmaRows * kp);
  p.b_lo = umma_align(p.b_hi + 4 * (size_t)nb_rows * kp);
  p.stage = umma_align(p.b_lo + 4 * (size_t)nb_rows * kp);
  p.total = umma_align(p.stage + 2 * 4 * (size_t)kUmmaRows * N);
  return p;
}

// Persistent CTAs walk the work list (pair, A group, 128-row tile) with a stride of the grid.
// Per work item: the A tile and the group's slices arrive by bulk copies on bar_ld (requested
// while the previous item was being finished), are split into the operand buffers, the raw
// buffers are refilled for the next item at once, one thread issues the MMAs (one pass of up to
// `ncols` accumulator columns at a time), and each item's 128 x N result goes from tensor memory
// through one of two staging tiles to global memory by a bulk store (direct stores when the
// output is not 16-byte aligned).
template <int NA>
__global__ void __launch_bounds__(128) level_umma_kernel(GemmDesc g, int rtiles, int kp,
                                                         int sb_max, int nb_rows, int ncols,
                                                         int et, int bulk_out,
                                                         long long n_work,
                                                         const __grid_constant__ CUtensorMap tmA,
                                                         int use_tmap) {
  extern __shared__ __align__(128) unsigned char usm[];
  __shared__ __align__(8) unsigned long long bar_ld;
  __shared__ __align__(8) unsigned long long bar_mma;
  __shared__ unsigned tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = g.K, N = g.N;
  const unsigned sbo = 32u * (unsigned)kp;
  const int nk4 = (N * K + 3) & ~3;
  const UmmaLevelSmem L = umma_level_plan(K, kp, N, sb_max, nb_rows);
  float* As = reinterpret_cast<float*>(usm + L.raw_a);
  float* Er = reinterpret_cast<float*>(usm + L.raw_e);
  uint32_t* Ah = reinterpret_cast<uint32_t*>(usm + L.a_hi);
  uint32_t* Al = reinterpret_cast<uint32_t*>(usm + L.a_lo);
  uint32_t* Bh = reinterpret_cast<uint32_t*>(usm + L.b_hi);
  uint32_t* Bl = reinterpret_cast<uint32_t*>(usm + L.b_lo);
  float* stage = reinterpret_cast<float*>(usm + L.stage);

  if (tid == 0) {
    mbar_init(&bar_ld, 1);
    mbar_init(&bar_mma, 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  // work item -> (pair, group, row tile)
  auto decode = [&](long long w, int& pair, int& q, int& r0, int& nrow) {
    const int rt = (int)(w % rtiles);
    const long long rest = w / rtiles;
    q = (int)(rest % g.st.n_grp);
    pair = (int)(rest / g.st.n_grp);
    r0 = rt * kUmmaRows;
    nrow = min(kUmmaRows, g.M - r0);
  };
  auto request = [&](long long w) {   // thread 0: bulk copies of work item w
    int pair, q, r0, nrow;
    decode(w, pair, q, r0, nrow);
    const int gs = g.st.grp_ptr[q], ns = g.st.grp_ptr[q + 1] - gs;
    const float* Ab = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket) + g.st.grp_a[q] + r0;
    const float* Bb = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket);
    if (use_tmap && (smem_addr(As) & 127u) == 0u) {
      // the A tile as one tensor copy (a box of 128 x K of the buffer's row view)
      mbar_expect_tx(&bar_ld, (unsigned)(K * kUmmaRows + ns * N * K) * 4u);
      tensor_copy_g2s(As, &tmA, r0,
                      (int)((Ab - r0 - static_cast<const float*>(g.A.base)) / g.a_sk), &bar_ld);
    } else {
      mbar_expect_tx(&bar_ld, (unsigned)(K * nrow + ns * N * K) * 4u);
      for (int b = 0; b < K; ++b)
        bulk_copy_g2s(As + b * kUmmaRows, Ab + (long long)b * g.a_sk, nrow * 4u, &bar_ld);
    }
    for (int j = 0; j < ns; ++j)
      bulk_copy_g2s(Er + j * nk4, Bb + g.st.grp_b[gs + j], N * K * 4u, &bar_ld);
  };

  long long w = blockIdx.x;
  if (tid == 0 && w < n_work) request(w);
  unsigned ph_ld = 0, ph_mma = 0;
  bool ld_pending = w < n_work, mma_pending = false, failed = false;
  int n_stores = 0;   // bulk stores of this warp (its staging tile = n_stores % 2)
  const unsigned a_hi = smem_addr(Ah), a_lo = smem_addr(Al);
  const unsigned b_hi = smem_addr(Bh), b_lo = smem_addr(Bl);
  const int kq4 = kp >> 2;
  for (; w < n_work; w += gridDim.x) {
    int pair, q, r0, nrow;
    decode(w, pair, q, r0, nrow);
    const int gs = g.st.grp_ptr[q], ns = g.st.grp_ptr[q + 1] - gs;
    if (__syncthreads_or(!mbar_wait(&bar_ld, ph_ld, g.wait_flag))) {
      failed = true;
      break;
    }
    ph_ld ^= 1u;
    ld_pending = false;
    // split into the operand buffers (rows / columns past the data are zero)
    for (int kq = 0; kq < kq4; ++kq) {
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = 4 * kq + u;
        x[u] = (tid < nrow && b < K) ? As[b * kUmmaRows + tid] : 0.f;
      }
      umma_store_split(Ah, Al, tid, kq, kp, x);
    }
    for (int i = tid; i < nb_rows * kq4; i += kUmmaRows) {
      const int n = i / kq4, kq = i - n * kq4;
      const int j = n / NA, a = n - j * NA;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      if (j < ns && a < N) {
        const float* Ej = Er + j * nk4;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int b = 4 * kq + u;
          if (b < K) x[u] = et ? Ej[b * N + a] : Ej[a * K + b];
        }
      }
      umma_store_split(Bh, Bl, n, kq, kp, x);
    }
    fence_proxy_async();   // operands visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const long long wn = w + gridDim.x;
    if (tid == 0 && wn < n_work) {
      fence_proxy_async();   // raw buffers were read above; refill them for the next item
      request(wn);
    }
    ld_pending = wn < n_work;

    long long cidx = 0;
    if (g.c_mode == MODE_PAIR) cidx = pair;
    else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
    else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
    float* Cpair = static_cast<float*>(g.C) + cidx * g.c_pstride;
    const int ipp = ncols / NA;
    for (int j0 = 0; j0 < ns; j0 += ipp) {
      const int nj = min(ipp, ns - j0);
      if (tid == 0) {
        const uint32_t idesc = umma_idesc_tf32(kUmmaRows, (nj * NA + 15) & ~15);
        const unsigned boff = (unsigned)(j0 * NA / 8) * sbo;
        for (int ks = 0; ks < kp / 8; ++ks) {
          const unsigned ko = (unsigned)ks * 256u;   // two core matrices along K
          umma_tf32(tmem, umma_sdesc(a_lo + ko, sbo), umma_sdesc(b_hi + boff + ko, sbo), idesc,
                    ks > 0);
          umma_tf32(tmem, umma_sdesc(a_hi + ko, sbo), umma_sdesc(b_lo + boff + ko, sbo), idesc, 1);
          umma_tf32(tmem, umma_sdesc(a_hi + ko, sbo), umma_sdesc(b_hi + boff + ko, sbo), idesc, 1);
        }
        umma_commit(&bar_mma);
      }
      mma_pending = true;
      if (__syncthreads_or(
              !mbar_wait(&bar_mma, ph_mma, g.wait_flag, kWaitBudgetNs, TTN_WAIT_FLAG_MMA))) {
        failed = true;
        break;
      }
      ph_mma ^= 1u;
      mma_pending = false;
      tc_fence_after();
      const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
      for (int jj = 0; jj < nj; ++jj) {
        float v[NA];
        tmem_ld_row<NA>(lane_base + (unsigned)(jj * NA), v);
        umma_store_tile<NA>(Cpair + g.st.grp_c[gs + j0 + jj] + (long long)r0 * N, nrow, N, v,
                            stage + warp * 64 * N, n_stores, bulk_out);
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
    if (failed) break;
  }
  // leave only with nothing in flight that targets this CTA (bounded second waits)
  if (failed && ld_pending) mbar_wait(&bar_ld, ph_ld, nullptr, kWaitDrainNs);
  if (failed && mma_pending) mbar_wait(&bar_mma, ph_mma, nullptr, kWaitDrainNs);
  if ((tid & 31) == 0) bulk_store_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// Segmented level stage on the tensor cores: Z[item] = sum_seg A_seg x E_seg (the operator-first
// last level, items = slots, segments = (prefix, slot) groups), one 128-row tile of one item per
// work item, persistent CTAs striding over the work list. The CTA walks its segments in order
// through two raw stages (A tile + slice by bulk copies, requested two segments ahead) and two
// operand buffers (the hi/lo split of a segment is written while the MMAs of the previous one
// run; a buffer is rewritten only after the MMAs that read it have completed, mma_done[b]). All
// segments of an item accumulate into one float32 accumulator of roundup16(NA) tensor-memory
// columns; the finished tile goes out through a staging tile and a bulk store (direct stores
// when the output is not 16-byte aligned). Items without segments are written as zeros.
struct UmmaSegSmem {
  // buffer b of a kind starts at <kind> + b * <kind>_stride
  size_t raw, raw_stride, op, op_stride, a_lo, b_hi, b_lo;   // a_lo, b_hi, b_lo: within op
  size_t stage, total;
};
__host__ __device__ inline UmmaSegSmem umma_seg_plan(int K, int kp, int N, int nb_rows) {
  UmmaSegSmem p;
  const size_t nk4 = (size_t)((N * K + 3) & ~3);
  p.raw = 0;
  p.raw_stride = umma_align(4 * ((size_t)K * kUmmaRows + nk4));
  p.op = 2 * p.raw_stride;
  p.a_lo = umma_align(4 * (size_t)kUmmaRows * kp);
  p.b_hi = umma_align(p.a_lo + 4 * (size_t)kUmmaRows * kp);
  p.b_lo = umma_align(p.b_hi + 4 * (size_t)nb_rows * kp);
  p.op_stride = umma_align(p.b_lo + 4 * (size_t)nb_rows * kp);
  p.stage = p.op + 2 * p.op_stride;
  p.total = umma_align(p.stage + 2 * 4 * (size_t)kUmmaRows * N);
  return p;
}

template <int NA>
__global__ void __launch_bounds__(128) level_umma_seg_kernel(GemmDesc g, int rtiles, int kp,
                                                             int et, int bulk_out,
                                                             long long n_work,
                                                             const __grid_constant__ CUtensorMap tmA,
                                                             int use_tmap) {
  constexpr int NB = (NA + 15) & ~15;   // B rows = accumulator columns
  constexpr int kCols = 32;             // tensor-memory allocation (>= NB, a power of two)
  static_assert(NB <= kCols, "accumulator wider than its allocation");
  extern __shared__ __align__(128) unsigned char usm[];
  __shared__ __align__(8) unsigned long long full[2];
  __shared__ __align__(8) unsigned long long mma_done[2];
  __shared__ unsigned tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = g.K, N = g.N;
  const unsigned sbo = 32u * (unsigned)kp;
  const int nk4 = (N * K + 3) & ~3;
  const int kq4 = kp >> 2;
  const UmmaSegSmem L = umma_seg_plan(K, kp, N, NB);
  float* stage = reinterpret_cast<float*>(usm + L.stage);

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&mma_done[b], 1);
    }
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  auto decode = [&](long long w, int& pair, int& sub, int& r0, int& nrow) {
    const int rt = (int)(w % rtiles);
    const long long rest = w / rtiles;
    sub = (int)(rest % g.st.n_sub);
    pair = (int)(rest / g.st.n_sub);
    r0 = rt * kUmmaRows;
    nrow = min(kUmmaRows, g.M - r0);
  };
  auto nseg_of = [&](long long w) {
    const int sub = (int)((w / rtiles) % g.st.n_sub);
    return g.st.seg_ptr[sub + 1] - g.st.seg_ptr[sub];
  };
  // thread 0's request cursor: the next segment (work item rq_w, segment rq_s) to bulk-copy
  long long rq_w = blockIdx.x;
  int rq_s = 0;
  auto skip_empty = [&]() {
    while (rq_w < n_work && nseg_of(rq_w) == 0) rq_w += gridDim.x;
  };
  auto request = [&](int b) {   // thread 0: copies of the cursor's segment into raw stage b
    if (rq_w >= n_work) return false;
    int pair, sub, r0, nrow;
    decode(rq_w, pair, sub, r0, nrow);
    const int sg = g.st.seg_ptr[sub] + rq_s;
    float* As = reinterpret_cast<float*>(usm + L.raw + b * L.raw_stride);
    float* Es = As + K * kUmmaRows;
    const float* Ab = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket) + g.st.seg_a[sg] + r0;
    const float* Bb = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket) + g.st.seg_b[sg];
    if (use_tmap && (smem_addr(As) & 127u) == 0u) {
      mbar_expect_tx(&full[b], (unsigned)(K * kUmmaRows + N * K) * 4u);
      tensor_copy_g2s(As, &tmA, r0,
                      (int)((Ab - r0 - static_cast<const float*>(g.A.base)) / g.a_sk), &full[b]);
    } else {
      mbar_expect_tx(&full[b], (unsigned)(K * nrow + N * K) * 4u);
      for (int kb = 0; kb < K; ++kb)
        bulk_copy_g2s(As + kb * kUmmaRows, Ab + (long long)kb * g.a_sk, nrow * 4u, &full[b]);
    }
    bulk_copy_g2s(Es, Bb, N * K * 4u, &full[b]);
    if (++rq_s == nseg_of(rq_w)) {
      rq_s = 0;
      rq_w += gridDim.x;
      skip_empty();
    }
    return true;
  };
  int n_req = 0;   // segments requested (thread 0)
  if (tid == 0) {
    skip_empty();
    if (request(0)) ++n_req;
    if (request(1)) ++n_req;
  }

  long long t = 0;   // segments consumed by this CTA
  bool failed = false;
  int n_stores = 0;   // bulk stores of this warp (its staging tile = n_stores % 2)
  for (long long w = blockIdx.x; w < n_work && !failed; w += gridDim.x) {
    int pair, sub, r0, nrow;
    decode(w, pair, sub, r0, nrow);
    const int s0 = g.st.seg_ptr[sub], nseg = g.st.seg_ptr[sub + 1] - s0;
    long long cidx = 0;
    if (g.c_mode == MODE_PAIR) cidx = pair;
    else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
    else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
    float* o = static_cast<float*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub] + (long long)r0 * N;
    for (int s = 0; s < nseg; ++s, ++t) {
      const int b = (int)(t & 1);
      bool ok = mbar_wait(&full[b], (unsigned)((t >> 1) & 1), g.wait_flag);
      if (ok && t >= 2)
        ok = mbar_wait(&mma_done[b], (unsigned)(((t >> 1) - 1) & 1), g.wait_flag, kWaitBudgetNs,
                       TTN_WAIT_FLAG_MMA);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      const float* As = reinterpret_cast<const float*>(usm + L.raw + b * L.raw_stride);
      const float* Es = As + K * kUmmaRows;
      unsigned char* op = usm + L.op + b * L.op_stride;
      uint32_t* Ah = reinterpret_cast<uint32_t*>(op);
      uint32_t* Al = reinterpret_cast<uint32_t*>(op + L.a_lo);
      uint32_t* Bh = reinterpret_cast<uint32_t*>(op + L.b_hi);
      uint32_t* Bl = reinterpret_cast<uint32_t*>(op + L.b_lo);
      for (int kq = 0; kq < kq4; ++kq) {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kb = 4 * kq + u;
          x[u] = (tid < nrow && kb < K) ? As[kb * kUmmaRows + tid] : 0.f;
        }
        umma_store_split(Ah, Al, tid, kq, kp, x);
      }
      for (int i = tid; i < NB * kq4; i += kUmmaRows) {
        const int n = i / kq4, kq = i - n * kq4;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (n < N) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int kb = 4 * kq + u;
            if (kb < K) x[u] = et ? Es[kb * N + n] : Es[n * K + kb];
          }
        }
        umma_store_split(Bh, Bl, n, kq, kp, x);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        fence_proxy_async();   // raw stage b was read above; refill it two segments ahead
        if (request(b)) ++n_req;
        const uint32_t idesc = umma_idesc_tf32(kUmmaRows, NB);
        const unsigned ah = smem_addr(Ah), al = smem_addr(Al);
        const unsigned bh = smem_addr(Bh), bl = smem_addr(Bl);
        for (int ks = 0; ks < kp / 8; ++ks) {
          const unsigned ko = (unsigned)ks * 256u;
          umma_tf32(tmem, umma_sdesc(al + ko, sbo), umma_sdesc(bh + ko, sbo), idesc,
                    (s > 0 || ks > 0) ? 1 : 0);
          umma_tf32(tmem, umma_sdesc(ah + ko, sbo), umma_sdesc(bl + ko, sbo), idesc, 1);
          umma_tf32(tmem, umma_sdesc(ah + ko, sbo), umma_sdesc(bh + ko, sbo), idesc, 1);
        }
        umma_commit(&mma_done[b]);
      }
    }
    if (failed) break;
    float v[NA];
    if (nseg > 0) {
      const int b = (int)((t - 1) & 1);
      if (__syncthreads_or(!mbar_wait(&mma_done[b], (unsigned)(((t - 1) >> 1) & 1), g.wait_flag,
                                      kWaitBudgetNs, TTN_WAIT_FLAG_MMA))) {
        failed = true;
        break;
      }
      tc_fence_after();
      tmem_ld_row<NA>(tmem + ((unsigned)(warp * 32) << 16), v);
    } else {
#pragma unroll
      for (int c = 0; c < NA; ++c) v[c] = 0.f;
    }
    umma_store_tile<NA>(o, nrow, N, v, stage + warp * 64 * N, n_stores, bulk_out);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // leave only with nothing in flight that targets this CTA (bounded second waits)
  if (failed && tid == 0) {
    for (long long u = t; u < n_req; ++u)
      mbar_wait(&full[u & 1], (unsigned)((u >> 1) & 1), nullptr, kWaitDrainNs);
    if (t > 0) mbar_wait(&mma_done[(t - 1) & 1], (unsigned)(((t - 1) >> 1) & 1), nullptr,
                         kWaitDrainNs);
  }
  if ((tid & 31) == 0) bulk_store_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
  }
}

namespace {
int level_tma_na(int N) { return N <= 8 ? 8 : N <= 16 ? 16 : N <= 24 ? 24 : N <= 32 ? 32 : 0; }
int level_tma_rows(int M) {
  const int nwt = (M + 31) / 32;
  const int ncta = (nwt + 8) / 9;
  return (nwt + ncta - 1) / ncta * 32;
}
// row tile of at most maxw warps, the tiles of M as even as whole warps allow
int level_tma_rows_cap(int M, int maxw) {
  const int nwt = (M + 31) / 32;
  const int ncta = (nwt + maxw - 1) / maxw;
  return (nwt + ncta - 1) / ncta * 32;
}
int level_env_floats_host(int NA, bool tc, int K) { return tc ? 2 * NA * (K + 4) : K * NA; }
size_t level_tma_smem_rows(int rows, int N, int K, int sb, bool tc) {
  const int na = level_tma_na(N);
  const int lda = rows + (tc ? 8 : 0);
  return sizeof(float) * ((size_t)K * lda + (size_t)sb * ((N * K + 3) & ~3) +
                          (size_t)sb * level_env_floats_host(na, tc, K));
}
size_t level_tma_smem(int M, int N, int K, int sb, bool tc) {
  const int na = level_tma_na(N);
  const int lda = level_tma_rows(M) + (tc ? 8 : 0);
  return sizeof(float) * ((size_t)K * lda + (size_t)sb * ((N * K + 3) & ~3) +
                          (size_t)sb * level_env_floats_host(na, tc, K));
}
size_t level_tma_seg_smem(int M, int N, int K, bool tc) {
  const int na = level_tma_na(N);
  const int lda = level_tma_rows(M) + (tc ? 8 : 0);
  return sizeof(float) * 2 *
         ((size_t)K * lda + (size_t)((N * K + 3) & ~3) + (size_t)level_env_floats_host(na, tc, K));
}
constexpr size_t kLevelTmaSmem = 100 * 1024;
}  // namespace

// The cap holds for both compute layouts (the tensor-core layout is the larger one).
int level_group_cap(int M, int N, int K) {
  if (M <= 0 || M % 4 != 0 || K <= 0 || K > 64 || (N * K) % 4 != 0 || level_tma_na(N) == 0)
    return 0;
  for (int sb = 6; sb >= 1; --sb)
    if (level_tma_smem(M, N, K, sb, true) <= kLevelTmaSmem) return sb;
  return 0;
}

// True if a float32 level launch meets the bulk-copy kernel's layout and alignment needs: A rows
// contiguous with a 16-byte aligned start for every (base, segment, k), E slices contiguous and
// aligned, A groups present.
static bool level_tma_ok(const GemmDesc& g) {
  if (level_group_cap(g.M, g.N, g.K) <= 0) return false;
  if (g.st.n_grp <= 0 && level_tma_seg_smem(g.M, g.N, g.K, true) > kLevelTmaSmem) return false;
  const bool e_ab = g.b_sk == 1 && g.b_sn == g.K;   // slices stored [a][b]
  const bool e_ba = g.b_sn == 1 && g.b_sk == g.N;   // slices stored [b][a]
  if (g.a_sm != 1 || g.a_sk % 4 != 0 || !(e_ab || e_ba) || g.c_sm != g.N || g.c_sn != 1)
    return false;
  if (g.A.pstride % 4 != 0 || g.B.pstride % 4 != 0) return false;
  if (reinterpret_cast<uintptr_t>(g.A.base) % 16 || reinterpret_cast<uintptr_t>(g.B.base) % 16)
    return false;
  return g.hst->a4 && g.hst->b4;
}

// Tensor map of a level stage's A operand (K slices of a_sk contiguous floats per item) as a
// row view of its buffer, boxes of box_x x K: only where every item's block starts a row of the
// buffer and the buffer holds whole rows.
static bool level_a_tensor_map(const GemmDesc& g, int box_x, CUtensorMap* tm) {
  if (box_x > 256 || g.K > 256 || g.a_sm != 1 || g.a_sk <= 0 || g.a_len % g.a_sk) return false;
  if (g.A.mode != MODE_CONST && g.A.pstride % g.a_sk) return false;
  for (long long a : g.hst->seg_a)
    if (a % g.a_sk) return false;
  for (long long a : g.hst->grp_a)
    if (a % g.a_sk) return false;
  return make_row_tensor_map(tm, g.A.base, g.a_sk, g.a_len / g.a_sk, box_x, g.K);
}

// Tensor-memory columns of one CTA of the tensor-core grouped level stage: the group's items
// (NA columns each) rounded up to a power of two, at most 128 (larger groups take passes), so
// that up to four CTAs can share an SM's 512 columns.
static int umma_level_cols(int sb_max, int na) {
  const int need = (sb_max * na + 15) & ~15;
  int c = 32;
  while (c < need && c < 128) c *= 2;
  return c;
}

// The tensor-core grouped level stage takes A-group launches the bulk-copy kernel takes, with
// N <= 32 and K <= 64 (any K: the padding to a multiple of 8 is zero).
static bool umma_level_ok(const GemmDesc& g) {
  if (g.st.n_grp <= 0 || g.K > 64 || level_tma_na(g.N) == 0 || !level_tma_ok(g)) return false;
  const int na = level_tma_na(g.N), kp = (g.K + 7) & ~7;
  return umma_level_plan(g.K, kp, g.N, g.hst->grp_max, g.hst->grp_max * na + 8).total <=
         200 * 1024;
}

// Dynamic shared memory for a launch of `kern` with `need` bytes, and the CTAs per SM it allows.
// Shared memory bounds the CTAs an SM can hold at floor(smem per SM / (bytes + reserved per
// CTA)); the request is padded until that bound times `ncols` is at most the 512 tensor-memory
// columns of an SM, so that every resident CTA's tcgen05.alloc finds free columns. The kernel
// prefers the largest shared-memory carveout, and the persistent grid is SMs x that bound.
static std::pair<size_t, int> umma_launch_smem(const void* kern, size_t need, int ncols,
                                               int device) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, size_t, int, int>, std::pair<size_t, int>> memo;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(kern, need, ncols, device);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  int optin = 0, per_sm = 0, reserved = 0;
  CUDA_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  CUDA_CHECK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  CUDA_CHECK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
  cudaFuncAttributes fa{};
  CUDA_CHECK(cudaFuncGetAttributes(&fa, kern));
  const size_t dyn_max = (size_t)optin - fa.sharedSizeBytes;
  TTN_REQUIRE(need <= dyn_max, "tensor-core level kernel: %zu bytes of shared memory needed",
              need);
  CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
  CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
  auto fit = [&](size_t sm) {
    return (int)((size_t)per_sm / (sm + fa.sharedSizeBytes + (size_t)reserved));
  };
  size_t sm = need;
  while (fit(sm) * ncols > 512) {
    sm += 1024;
    TTN_REQUIRE(sm <= dyn_max, "tensor-core level kernel: cannot bound CTAs per SM");
  }
  const int resident = fit(sm);
  TTN_REQUIRE(resident >= 1, "tensor-core level kernel: does not fit on an SM");
  memo[key] = {sm, resident};
  return memo[key];
}

// The tensor-core segmented level stage takes the launches of the segmented bulk-copy path
// (items summing several segments), with N <= 32 and K <= 64.
static bool umma_seg_ok(const GemmDesc& g) {
  if (g.st.n_grp > 0 || g.K > 64 || level_tma_na(g.N) == 0 || !level_tma_ok(g)) return false;
  const int kp = (g.K + 7) & ~7;
  return umma_seg_plan(g.K, kp, g.N, (level_tma_na(g.N) + 15) & ~15).total <= 200 * 1024;
}

static void launch_level_umma_seg(ttn_ctx* ctx, const GemmDesc& g) {
  const int na = level_tma_na(g.N);
  const int kp = (g.K + 7) & ~7;
  const size_t need = umma_seg_plan(g.K, kp, g.N, (na + 15) & ~15).total;
  const int rt = (g.M + kUmmaRows - 1) / kUmmaRows;
  const long long n_work = (long long)rt * g.st.n_sub * g.n_pairs;
  const bool bulk_out = g.N % 4 == 0 && g.c_pstride % 4 == 0 &&
                        reinterpret_cast<uintptr_t>(g.C) % 16 == 0 && g.hst->c4;
  const bool et = g.b_sn == 1 && g.b_sk == g.N && g.K != 1;
  const double flops = 2.0 * g.M * g.N * (double)g.K * g.hst->n_seg * g.n_pairs;
  static const char* nm[] = {"level_tc05_seg_8", "level_tc05_seg_16", "level_tc05_seg_24",
                             "level_tc05_seg_32"};
  LaunchScope ls(ctx, nm[na / 8 - 1], flops, algorithmic_bytes(g, sizeof(float)));
  GemmDesc gd = g;
  gd.wait_flag = ctx->d_wait;
  CUtensorMap tmA{};
  const bool tmap = level_a_tensor_map(g, kUmmaRows, &tmA);
  auto go = [&](auto kern) {
    const auto [sm, resident] = umma_launch_smem((const void*)kern, need, 32, ctx->device);
    const long long grid = std::min<long long>(n_work, (long long)ctx->sm_count * resident);
    kern<<<(unsigned)grid, kUmmaRows, sm, ctx->stream>>>(gd, rt, kp, et ? 1 : 0,
                                                         bulk_out ? 1 : 0, n_work, tmA,
                                                         tmap ? 1 : 0);
  };
  switch (na) {
    case 8: go(level_umma_seg_kernel<8>); break;
    case 16: go(level_umma_seg_kernel<16>); break;
    case 24: go(level_umma_seg_kernel<24>); break;
    default: go(level_umma_seg_kernel<32>); break;
  }
  CUDA_LAUNCH_CHECK();
}

static void launch_level_umma(ttn_ctx* ctx, const GemmDesc& g) {
  const int na = level_tma_na(g.N);
  const int kp = (g.K + 7) & ~7;
  const int sb_max = g.hst->grp_max;
  const int nb_rows = sb_max * na + 8;
  const int ncols = umma_level_cols(sb_max, na);
  const size_t need = umma_level_plan(g.K, kp, g.N, sb_max, nb_rows).total;
  const int rt = (g.M + kUmmaRows - 1) / kUmmaRows;
  const long long n_work = (long long)rt * g.st.n_grp * g.n_pairs;
  const bool bulk_out = g.N % 4 == 0 && g.c_pstride % 4 == 0 &&
                        reinterpret_cast<uintptr_t>(g.C) % 16 == 0 && g.hst->c4;
  const bool et = g.b_sn == 1 && g.b_sk == g.N && g.K != 1;
  const double flops = 2.0 * g.M * g.N * (double)g.K * g.st.n_sub * g.n_pairs;
  static const char* nm[] = {"level_tc05_8", "level_tc05_16", "level_tc05_24", "level_tc05_32"};
  LaunchScope ls(ctx, nm[na / 8 - 1], flops, algorithmic_bytes(g, sizeof(float)));
  GemmDesc gd = g;
  gd.wait_flag = ctx->d_wait;
  CUtensorMap tmA{};
  const bool tmap = level_a_tensor_map(g, kUmmaRows, &tmA);
  auto go = [&](auto kern) {
    const auto [sm, resident] = umma_launch_smem((const void*)kern, need, ncols, ctx->device);
    const long long grid = std::min<long long>(n_work, (long long)ctx->sm_count * resident);
    kern<<<(unsigned)grid, kUmmaRows, sm, ctx->stream>>>(gd, rt, kp, sb_max, nb_rows, ncols,
                                                         et ? 1 : 0, bulk_out ? 1 : 0, n_work,
                                                         tmA, tmap ? 1 : 0);
  };
  switch (na) {
    case 8: go(level_umma_kernel<8>); break;
    case 16: go(level_umma_kernel<16>); break;
    case 24: go(level_umma_kernel<24>); break;
    default: go(level_umma_kernel<32>); break;
  }
  CUDA_LAUNCH_CHECK();
}

template <class T>
void launch_level(ttn_ctx* ctx, const GemmDesc& g) {
  if (g.n_pairs <= 0 || g.st.n_sub <= 0 || g.M <= 0 || g.N <= 0) return;
  TTN_REQUIRE(level_shape_ok(g), "level kernel: unsupported shape");
  check_bounds(g, sizeof(T));
  // TTN_TF32X3: tensor-core compute on the staged tiles (K a multiple of 8)
  const bool tc = sizeof(T) == 4 && ctx->tf32x3 && g.K % 8 == 0;
  if (sizeof(T) == 4 && ctx->tf32x3 && !(tc && level_tma_ok(g)) && level_tc_ok(g)) {
    launch_level_tc(ctx, g);
    return;
  }
  if (sizeof(T) == 4 && ctx->tc05 && umma_seg_ok(g)) {
    launch_level_umma_seg(ctx, g);
    return;
  }
  if (sizeof(T) == 4 && level_tma_ok(g) && g.st.n_grp == 0) {
    // items with several segments: one CTA per (pair, item, row tile), segments through a ring
    const int na = level_tma_na(g.N);
    const int rows_cta = level_tma_rows(g.M);
    const int rt = (g.M + rows_cta - 1) / rows_cta;
    const size_t smem = level_tma_seg_smem(g.M, g.N, g.K, tc);
    bool vec = g.N == na && g.c_pstride % 2 == 0 &&
               reinterpret_cast<uintptr_t>(g.C) % 8 == 0;
    vec = vec && g.hst->c2;
    const long long grid = (long long)rt * g.st.n_sub * g.n_pairs;
    TTN_REQUIRE(grid <= 0x7fffffffLL, "level grid too large");
    const double flops = 2.0 * g.M * g.N * (double)g.K * g.hst->n_seg * g.n_pairs;
    static const char* nm[] = {"level_tma_seg_f32_8", "level_tma_seg_f32_16",
                               "level_tma_seg_f32_24", "level_tma_seg_f32_32"};
    static const char* nm_tc[] = {"level_tma_seg_tf32x3_8", "level_tma_seg_tf32x3_16",
                                  "level_tma_seg_tf32x3_24", "level_tma_seg_tf32x3_32"};
    LaunchScope ls(ctx, (tc ? nm_tc : nm)[na / 8 - 1], flops, algorithmic_bytes(g, sizeof(T)));
    GemmDesc gd = g;
    gd.wait_flag = ctx->d_wait;
    const bool et = g.b_sn == 1 && g.b_sk == g.N && g.K != 1;
    if (et && g.N == na) {
      // slices already in the SIMT compute layout: warp-specialised copy/compute pipeline
      // (float32 SIMT, or 3xTF32 tensor cores with A rows padded by 8 floats). Where the A
      // buffer has a tensor-map row view, tiles of at most 8 warps (the box holds at most 256
      // columns) come as one tensor copy each.
      CUtensorMap tmA{};
      int rows_ws = level_tma_rows_cap(g.M, 8);
      const bool tmap = level_a_tensor_map(g, rows_ws + (tc ? 8 : 0), &tmA);
      if (!tmap) rows_ws = rows_cta;
      const int rt_ws = (g.M + rows_ws - 1) / rows_ws;
      const long long grid_ws = (long long)rt_ws * g.st.n_sub * g.n_pairs;
      TTN_REQUIRE(grid_ws <= 0x7fffffffLL, "level grid too large");
      const int lda = rows_ws + (tc ? 8 : 0);
      const size_t smem_ws = sizeof(float) * 2 * (size_t)seg_ws_stage_floats(g.K, lda, na);
      auto go_ws = [&](auto kern) {
        smem_attr((const void*)kern, (int)kLevelTmaSmem, ctx->device);
        kern<<<(unsigned)grid_ws, rows_ws + 32, smem_ws, ctx->stream>>>(gd, rt_ws, rows_ws,
                                                                          vec ? 1 : 0, tmA);
      };
      auto pick = [&](auto t_tc, auto t_map) {
        constexpr bool TCv = decltype(t_tc)::value, TMv = decltype(t_map)::value;
        switch (na) {
          case 8: go_ws(level_seg_ws_kernel<8, TCv, TMv>); break;
          case 16: go_ws(level_seg_ws_kernel<16, TCv, TMv>); break;
          case 24: go_ws(level_seg_ws_kernel<24, TCv, TMv>); break;
          default: go_ws(level_seg_ws_kernel<32, TCv, TMv>); break;
        }
      };
      using T_ = std::true_type;
      using F_ = std::false_type;
      if (tc) tmap ? pick(T_{}, T_{}) : pick(T_{}, F_{});
      else tmap ? pick(F_{}, T_{}) : pick(F_{}, F_{});
      CUDA_LAUNCH_CHECK();
      return;
    }
    auto go = [&](auto kern) {
      smem_attr((const void*)kern, (int)kLevelTmaSmem, ctx->device);
      kern<<<(unsigned)grid, rows_cta, smem, ctx->stream>>>(gd, rt, rows_cta, vec ? 1 : 0,
                                                            et ? 1 : 0);
    };
    if (tc) {
      switch (na) {
        case 8: go(level_tma_seg_kernel<8, true>); break;
        case 16: go(level_tma_seg_kernel<16, true>); break;
        case 24: go(level_tma_seg_kernel<24, true>); break;
        default: go(level_tma_seg_kernel<32, true>); break;
      }
    } else {
      switch (na) {
        case 8: go(level_tma_seg_kernel<8, false>); break;
        case 16: go(level_tma_seg_kernel<16, false>); break;
        case 24: go(level_tma_seg_kernel<24, false>); break;
        default: go(level_tma_seg_kernel<32, false>); break;
      }
    }
    CUDA_LAUNCH_CHECK();
    return;
  }
  if (sizeof(T) == 4 && ctx->tc05 && umma_level_ok(g)) {
    launch_level_umma(ctx, g);
    return;
  }
  if (sizeof(T) == 4 && level_tma_ok(g)) {
    const int na = level_tma_na(g.N);
    // tiles of at most 8 warps with the A tile as one tensor copy where the A buffer has a
    // tensor-map row view (a box holds at most 256 columns), else up to 9 warps and row copies
    CUtensorMap tmA{};
    int rows_cta = level_tma_rows_cap(g.M, 8);
    const bool tmap = level_a_tensor_map(g, rows_cta + (tc ? 8 : 0), &tmA);
    if (!tmap) rows_cta = level_tma_rows(g.M);
    const int rt = (g.M + rows_cta - 1) / rows_cta;
    const int sb_max = g.hst->grp_max;
    const size_t smem = level_tma_smem_rows(rows_cta, g.N, g.K, sb_max, tc);
    TTN_REQUIRE(smem <= kLevelTmaSmem, "level kernel: A group larger than its cap");
    bool vec = g.N == na && g.c_pstride % 2 == 0 &&
               reinterpret_cast<uintptr_t>(g.C) % 8 == 0;
    vec = vec && g.hst->c2;
    const long long grid = (long long)rt * g.st.n_grp * g.n_pairs;
    TTN_REQUIRE(grid <= 0x7fffffffLL, "level grid too large");
    const double flops = 2.0 * g.M * g.N * (double)g.K * g.st.n_sub * g.n_pairs;
    static const char* nm[] = {"level_tma_f32_8", "level_tma_f32_16", "level_tma_f32_24",
                               "level_tma_f32_32"};
    static const char* nm_tc[] = {"level_tma_tf32x3_8", "level_tma_tf32x3_16",
                                  "level_tma_tf32x3_24", "level_tma_tf32x3_32"};
    LaunchScope ls(ctx, (tc ? nm_tc : nm)[na / 8 - 1], flops, algorithmic_bytes(g, sizeof(T)));
    GemmDesc gd = g;
    gd.wait_flag = ctx->d_wait;
    const int threads = rows_cta;   // 32 rows per warp
    auto go = [&](auto kern) {
      smem_attr((const void*)kern, (int)kLevelTmaSmem, ctx->device);
      const bool et = g.b_sn == 1 && g.b_sk == g.N && g.K != 1;
      kern<<<(unsigned)grid, threads, smem, ctx->stream>>>(gd, rt, rows_cta, sb_max, vec ? 1 : 0,
                                                           et ? 1 : 0, tmA);
    };
    auto pick = [&](auto t_tc, auto t_map) {
      constexpr bool TCv = decltype(t_tc)::value, TMv = decltype(t_map)::value;
      switch (na) {
        case 8: go(level_tma_kernel<8, TCv, TMv>); break;
        case 16: go(level_tma_kernel<16, TCv, TMv>); break;
        case 24: go(level_tma_kernel<24, TCv, TMv>); break;
        default: go(level_tma_kernel<32, TCv, TMv>); break;
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (tc) tmap ? pick(T_{}, T_{}) : pick(T_{}, F_{});
    else tmap ? pick(F_{}, T_{}) : pick(F_{}, F_{});
    CUDA_LAUNCH_CHECK();
    return;
  }
  const int rtiles = (g.M + kThreads - 1) / kThreads;
  const long long grid = (long long)rtiles * g.st.n_sub * g.n_pairs;
  TTN_REQUIRE(grid <= 0x7fffffffLL, "level grid too large");
  long long nseg = 0;
  for (int q = 0; q < g.st.n_sub; ++q) nseg += g.hst->seg_ptr[q + 1] - g.hst->seg_ptr[q];
  const double flops = 2.0 * g.M * g.N * (double)g.K * nseg * g.n_pairs;
  const double bytes = algorithmic_bytes(g, sizeof(T));
  const int na = g.N <= 8 ? 8 : g.N <= 16 ? 16 : g.N <= 24 ? 24 : g.N <= 32 ? 32 : g.N <= 48 ? 48 : 64;
  static const char* n64[] = {"level_f64_8", "level_f64_16", "level_f64_24", "level_f64_32",
                              "level_f64_48", "level_f64_64"};
  static const char* n32[] = {"level_f32_8", "level_f32_16", "level_f32_24", "level_f32_32",
                              "level_f32_48", "level_f32_64"};
  const int ci = na == 8 ? 0 : na == 16 ? 1 : na == 24 ? 2 : na == 32 ? 3 : na == 48 ? 4 : 5;
  LaunchScope ls(ctx, sizeof(T) == 8 ? n64[ci] : n32[ci], flops, bytes);
  cudaStream_t s = ctx->stream;
  switch (na) {
    case 8: level_kernel<T, 8><<<grid, kThreads, 0, s>>>(g, rtiles); break;
    case 16: level_kernel<T, 16><<<grid, kThreads, 0, s>>>(g, rtiles); break;
    case 24: level_kernel<T, 24><<<grid, kThreads, 0, s>>>(g, rtiles); break;
    case 32: level_kernel<T, 32><<<grid, kThreads, 0, s>>>(g, rtiles); break;
    case 48: level_kernel<T, 48><<<grid, kThreads, 0, s>>>(g, rtiles); break;
    default: level_kernel<T, 64><<<grid, kThreads, 0, s>>>(g, rtiles); break;
  }
  CUDA_LAUNCH_CHECK();
}

__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  const double2 y = *reinterpret_cast<const double2*>(p + 2);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = y.x;
  v[3] = y.y;
}

// Closure stage of a node contraction, specialised for its shape: C[a][b] = sum_k A[a][k] Z[b][k]
// with a, b <= 32 and long k (A rows and Z rows contiguous in k). 256 threads = 4 groups that
// take interleaved 32-wide k chunks; inside a group an 8 x 8 thread grid owns 4 x 4 output
// tiles; shared tiles are k-major with a padded row (36) so 4-wide loads stay aligned; the four
// partial sums are reduced through shared memory at the end.
template <class T>
__global__ void __launch_bounds__(kThreads) closure_kernel(GemmDesc g) {
  constexpr int KC = sizeof(T) == 8 ? 16 : 32, LD = 36;
  static_assert(2 * 4 * KC * LD >= 4096, "reduction buffer");
  __shared__ __align__(16) T sh[2 * 4 * KC * LD];
  T(*As)[KC][LD] = reinterpret_cast<T(*)[KC][LD]>(sh);
  T(*Zs)[KC][LD] = reinterpret_cast<T(*)[KC][LD]>(sh + 4 * KC * LD);
  const int sub = (int)(blockIdx.x % g.st.n_sub);
  const int pair = (int)(blockIdx.x / g.st.n_sub);
  const int seg = g.st.seg_ptr[sub];
  const T* Ab = operand_base<T>(g.A, pair, g.pair_bra, g.pair_ket) + g.st.seg_a[seg];
  const T* Zb = operand_base<T>(g.B, pair, g.pair_bra, g.pair_ket) + g.st.seg_b[seg];
  const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int ty = t >> 3, tx = t & 7;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < g.K; k0 += 4 * KC) {
    // each thread loads for every group: 4 x (32 x 32) A values and the same for Z
    for (int i = threadIdx.x; i < 4 * KC * 32; i += kThreads) {
      const int gg = i / (KC * 32), rem = i % (KC * 32);
      const int row = rem / KC, kk = rem % KC;
      const int k = k0 + gg * KC + kk;
      As[gg][kk][row] = (row < g.M && k < g.K) ? Ab[(long long)row * g.a_sm + k] : T(0);
      Zs[gg][kk][row] = (row < g.N && k < g.K) ? Zb[(long long)row * g.b_sn + k] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      T a[4], b[4];
      load4(&As[grp][kk][ty * 4], a);   // 16-byte aligned: row stride 36, offset 4*ty
      load4(&Zs[grp][kk][tx * 4], b);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  // reduce the four groups (reuse the tiles as [4][32][32])
  T* red = sh;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) red[grp * 1024 + (ty * 4 + i) * 32 + tx * 4 + j] = acc[i][j];
  __syncthreads();
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  T* Cb = static_cast<T*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub];
  for (int i = threadIdx.x; i < 1024; i += kThreads) {
    const int a = i / 32, b = i % 32;
    if (a < g.M && b < g.N)
      Cb[(long long)a * g.c_sm + (long long)b * g.c_sn] =
          red[i] + red[1024 + i] + red[2048 + i] + red[3072 + i];
  }
}


// Shared-memory layout of one closure stage (floats): A rows at pitch ldk, then Z rows from the
// next 128-byte boundary, the stage rounded up to 128 bytes (tensor copies land 128-byte aligned).
__host__ __device__ inline int closure_z_offset(int mp, int ldk) { return (mp * ldk + 31) & ~31; }
__host__ __device__ inline int closure_stage_floats(int mp, int np, int ldk) {
  return (closure_z_offset(mp, ldk) + np * ldk + 31) & ~31;
}

// Closure GEMM with bulk-copied operands (float32): C[a][b] = sum_k A[a][k] Z[b][k] for one
// item per CTA, M, N <= MP, NP. K is cut into chunks of kc_max (a multiple of 8) that land in
// shared memory (rows padded to kc_max + 4 floats, so 16-byte loads of 8 consecutive rows hit
// distinct banks) through a two-stage ring of mbarrier-tracked bulk copies; chunk c + 2 is in
// flight while chunk c + 1 waits and chunk c is consumed. Each thread owns a TA x TB output tile
// and one of NS interleaved k-slices; the slice partials are summed in a fixed order through
// shared memory (aliasing the ring) at the end.
template <int TA, int TB, int MP, int NP, bool TMAP>
__global__ void __launch_bounds__(kThreads, 3)
    closure_tma_kernel(GemmDesc g, int kc_max, int nstage, const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmZ) {
  constexpr int NT = (MP / TA) * (NP / TB), NS = kThreads / NT;
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) unsigned long long bar[2];
  const int ldk = kc_max + 4;
  const int zoff = closure_z_offset(MP, ldk), stage = closure_stage_floats(MP, NP, ldk);
  const int sub = (int)(blockIdx.x % g.st.n_sub);
  const int pair = (int)(blockIdx.x / g.st.n_sub);
  const int seg = g.st.seg_ptr[sub];
  const float* Ab = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket) + g.st.seg_a[seg];
  const float* Zb = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket) + g.st.seg_b[seg];
  const int nchunk = (g.K + kc_max - 1) / kc_max;
  // first row of the item's A and Z blocks in the tensor maps' row view
  int ya = 0, yz = 0;
  if (TMAP && threadIdx.x == 0) {
    ya = (int)((Ab - static_cast<const float*>(g.A.base)) / g.a_sm);
    yz = (int)((Zb - static_cast<const float*>(g.B.base)) / g.b_sn);
  }
  auto issue = [&](int c, int s) {
    const int k0 = c * kc_max, kc = min(kc_max, g.K - k0);
    float* As = dsm + s * stage;
    float* Zs = As + zoff;
    if constexpr (TMAP) {
      // one box of (kc_max + 4) x M (x N) per operand: the rows land at pitch ldk, the 4 extra
      // columns (next row or zeros past the end) are never read. Tensor copies need 128-byte
      // aligned destinations: the row copies below stand in if the dynamic shared memory is not.
      if ((smem_addr(dsm) & 127u) == 0u) {
        mbar_expect_tx(&bar[s], (unsigned)((g.M + g.N) * ldk) * 4u);
        tensor_copy_g2s(As, &tmA, k0, ya, &bar[s]);
        tensor_copy_g2s(Zs, &tmZ, k0, yz, &bar[s]);
        return;
      }
    }
    mbar_expect_tx(&bar[s], (unsigned)((g.M + g.N) * kc) * 4u);
    for (int r = 0; r < g.M; ++r)
      bulk_copy_g2s(As + r * ldk, Ab + (long long)r * g.a_sm + k0, kc * 4u, &bar[s]);
    for (int r = 0; r < g.N; ++r)
      bulk_copy_g2s(Zs + r * ldk, Zb + (long long)r * g.b_sn + k0, kc * 4u, &bar[s]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    issue(0, 0);
    if (nchunk > 1) issue(1, 1);
  }
  const int tile = threadIdx.x % NT, ks = threadIdx.x / NT;
  const int ti = tile / (NP / TB), tj = tile % (NP / TB);
  float acc[TA][TB];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TB; ++j) acc[i][j] = 0.f;
  unsigned phase[2] = {0u, 0u};
  for (int c = 0; c < nchunk; ++c) {
    const int s = nstage == 2 ? (c & 1) : 0;
    const bool ok = mbar_wait(&bar[s], phase[s], g.wait_flag);
    phase[s] ^= 1u;
    if (__syncthreads_or(!ok)) return;
    const int kc = min(kc_max, g.K - c * kc_max);
    const float* As = dsm + s * stage;
    const float* Zs = As + zoff;
    if (ks < NS) {
      for (int qk = ks; qk < kc / 4; qk += NS) {
        const int k = qk * 4;
        float a[TA][4], b[TB][4];
#pragma unroll
        for (int i = 0; i < TA; ++i) load4(As + (ti * TA + i) * ldk + k, a[i]);
#pragma unroll
        for (int j = 0; j < TB; ++j) load4(Zs + (tj * TB + j) * ldk + k, b[j]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int i = 0; i < TA; ++i)
#pragma unroll
            for (int j = 0; j < TB; ++j) acc[i][j] = fmaf(a[i][u], b[j][u], acc[i][j]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && c + nstage < nchunk) {
      fence_proxy_async();
      issue(c + nstage, s);
    }
  }
  float* red = dsm;
  if (ks < NS) {
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) red[(ks * MP + ti * TA + i) * NP + tj * TB + j] = acc[i][j];
  }
  __syncthreads();
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  float* Cb = static_cast<float*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub];
  for (int i = threadIdx.x; i < MP * NP; i += kThreads) {
    const int a = i / NP, b = i % NP;
    if (a >= g.M || b >= g.N) continue;
    float v = 0.f;
    for (int q = 0; q < NS; ++q) v += red[q * MP * NP + i];
    Cb[(long long)a * g.c_sm + (long long)b * g.c_sn] = v;
  }
}

namespace {
constexpr size_t kClosureTmaSmem = 200 * 1024;
// chunk length (multiple of 8) and ring depth of the bulk-copy closure for contraction length K
void closure_tma_chunks(int K, int& kc_max, int& nstage) {
  if (K <= 256) {
    kc_max = (K + 7) & ~7;
    nstage = 1;
  } else {
    kc_max = 192;
    nstage = 2;
  }
}
int closure_tma_pad(const GemmDesc& g) {
  const int mn = std::max(g.M, g.N);
  return mn <= 12 ? 12 : mn <= 24 ? 24 : mn <= 32 ? 32 : 0;
}
size_t closure_tma_smem(int K, int pad) {
  int kc_max, nstage;
  closure_tma_chunks(K, kc_max, nstage);
  const int nt = pad == 12 ? 16 : pad == 24 ? 16 : 32;
  const size_t ring = (size_t)nstage * closure_stage_floats(pad, pad, kc_max + 4);
  const size_t red = (size_t)(kThreads / nt) * pad * pad;
  return sizeof(float) * std::max(ring, red);
}
}  // namespace

// Tensor maps of the closure operands (A rows of a_sm floats, Z rows of b_sn floats, boxes of
// kc_max + 4 columns): only where every item's block starts a row of its buffer (so a box never
// wraps into the next row's data at its start), the buffers hold whole rows and the box fits.
static bool closure_tensor_maps(const GemmDesc& g, int kc_max, CUtensorMap* tmA, CUtensorMap* tmZ) {
  const int box_x = kc_max + 4;
  if (box_x > 256 || g.M > 256 || g.N > 256 || g.a_sm <= 0 || g.b_sn <= 0) return false;
  if (g.a_len % g.a_sm || g.b_len % g.b_sn) return false;
  if ((g.A.mode != MODE_CONST && g.A.pstride % g.a_sm) ||
      (g.B.mode != MODE_CONST && g.B.pstride % g.b_sn))
    return false;
  for (long long a : g.hst->seg_a)
    if (a % g.a_sm) return false;
  for (long long b : g.hst->seg_b)
    if (b % g.b_sn) return false;
  return make_row_tensor_map(tmA, g.A.base, g.a_sm, g.a_len / g.a_sm, box_x, g.M) &&
         make_row_tensor_map(tmZ, g.B.base, g.b_sn, g.b_len / g.b_sn, box_x, g.N);
}

// True if a float32 closure launch meets the bulk-copy kernel's layout and alignment needs.
static bool closure_tma_ok(const GemmDesc& g) {
  const int pad = closure_tma_pad(g);
  if (pad == 0 || g.K <= 0 || g.K % 4 != 0 || g.a_sk != 1 || g.b_sk != 1) return false;
  if (g.a_sm % 4 != 0 || g.b_sn % 4 != 0 || g.A.pstride % 4 != 0 || g.B.pstride % 4 != 0)
    return false;
  if (reinterpret_cast<uintptr_t>(g.A.base) % 16 || reinterpret_cast<uintptr_t>(g.B.base) % 16)
    return false;
  if (!g.hst->a4 || !g.hst->b4) return false;
  return closure_tma_smem(g.K, pad) <= kClosureTmaSmem;
}


// Closure GEMM for short contractions (K <= 256) whose rows the bulk-copy kernel cannot take
// (K or the row starts not multiples of 4 floats, e.g. K = 81 or 9 on the chain nodes): both
// operand blocks (M x K and N x K) are loaded with coalesced element loads into shared rows of
// odd stride (conflict-free scalar loads of 8 rows of a tile), then TA x TB register tiles x NS
// interleaved k-slices as in closure_tma_kernel, slice partials summed in a fixed order.
template <class T, int TA, int TB, int MP, int NP>
__global__ void __launch_bounds__(kThreads, 3) closure_small_kernel(GemmDesc g, int ldk) {
  constexpr int NT = (MP / TA) * (NP / TB), NS = kThreads / NT;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  T* As = reinterpret_cast<T*>(dsm_raw);
  T* Zs = As + MP * ldk;
  const int sub = (int)(blockIdx.x % g.st.n_sub);
  const int pair = (int)(blockIdx.x / g.st.n_sub);
  const int seg = g.st.seg_ptr[sub];
  const T* Ab = operand_base<T>(g.A, pair, g.pair_bra, g.pair_ket) + g.st.seg_a[seg];
  const T* Zb = operand_base<T>(g.B, pair, g.pair_bra, g.pair_ket) + g.st.seg_b[seg];
  for (int i = threadIdx.x; i < g.M * g.K; i += kThreads) {
    const int r = i / g.K, k = i - r * g.K;
    As[r * ldk + k] = Ab[(long long)r * g.a_sm + k];
  }
  for (int i = threadIdx.x; i < g.N * g.K; i += kThreads) {
    const int r = i / g.K, k = i - r * g.K;
    Zs[r * ldk + k] = Zb[(long long)r * g.b_sn + k];
  }
  __syncthreads();
  const int tile = threadIdx.x % NT, ks = threadIdx.x / NT;
  const int ti = tile / (NP / TB), tj = tile % (NP / TB);
  T acc[TA][TB];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TB; ++j) acc[i][j] = T(0);
  if (ks < NS) {
    // rows past M / N hold stale shared memory; they only reach accumulators that are dropped
    for (int k = ks; k < g.K; k += NS) {
      T a[TA], b[TB];
#pragma unroll
      for (int i = 0; i < TA; ++i) a[i] = As[(ti * TA + i) * ldk + k];
#pragma unroll
      for (int j = 0; j < TB; ++j) b[j] = Zs[(tj * TB + j) * ldk + k];
#pragma unroll
      for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int j = 0; j < TB; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  __syncthreads();
  T* red = As;
  if (ks < NS) {
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) red[(ks * MP + ti * TA + i) * NP + tj * TB + j] = acc[i][j];
  }
  __syncthreads();
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  T* Cb = static_cast<T*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub];
  for (int i = threadIdx.x; i < MP * NP; i += kThreads) {
    const int a = i / NP, b = i % NP;
    if (a >= g.M || b >= g.N) continue;
    T v = T(0);
    for (int q = 0; q < NS; ++q) v += red[q * MP * NP + i];
    Cb[(long long)a * g.c_sm + (long long)b * g.c_sn] = v;
  }
}

namespace {
// shared bytes of closure_small_kernel: the two operand blocks, or the slice partials
size_t closure_small_smem(int K, int pad, size_t elem) {
  const int ldk = K | 1;
  const int nt = pad == 12 ? 16 : pad == 24 ? 16 : 32;
  const size_t ops = (size_t)2 * pad * ldk;
  const size_t red = (size_t)(kThreads / nt) * pad * pad;
  return elem * std::max(ops, red);
}
constexpr size_t kClosureSmallSmem = 96 * 1024;
}  // namespace

bool closure_shape_ok(const GemmDesc& g) {
  if (g.a_sk != 1 || g.b_sk != 1 || g.M > 32 || g.N > 32) return false;
  return g.hst->single;
}

template <class T>
void launch_closure(ttn_ctx* ctx, const GemmDesc& g) {
  if (g.n_pairs <= 0 || g.st.n_sub <= 0 || g.M <= 0 || g.N <= 0) return;
  TTN_REQUIRE(closure_shape_ok(g), "closure kernel: unsupported shape");
  check_bounds(g, sizeof(T));
  const long long grid = (long long)g.st.n_sub * g.n_pairs;
  TTN_REQUIRE(grid <= 0x7fffffffLL, "closure grid too large");
  const double flops = 2.0 * g.M * g.N * (double)g.K * g.st.n_sub * g.n_pairs;
  const double bytes = algorithmic_bytes(g, sizeof(T));
  const int pad_small = closure_tma_pad(g);
  if (sizeof(T) == 4 && !closure_tma_ok(g) && pad_small > 0 && g.K <= 256 &&
      closure_small_smem(g.K, pad_small, sizeof(T)) <= kClosureSmallSmem) {
    const int ldk = g.K | 1;
    const size_t smem = closure_small_smem(g.K, pad_small, sizeof(T));
    LaunchScope ls(ctx, "closure_small_f32", flops, bytes);
    auto go = [&](auto kern) {
      smem_attr((const void*)kern, (int)kClosureSmallSmem, ctx->device);
      kern<<<(unsigned)grid, kThreads, smem, ctx->stream>>>(g, ldk);
    };
    if (pad_small == 12) go(closure_small_kernel<float, 3, 3, 12, 12>);
    else if (pad_small == 24) go(closure_small_kernel<float, 6, 6, 24, 24>);
    else go(closure_small_kernel<float, 4, 8, 32, 32>);
    CUDA_LAUNCH_CHECK();
    return;
  }
  if (sizeof(T) == 4 && closure_tma_ok(g)) {
    const int pad = closure_tma_pad(g);
    int kc_max, nstage;
    closure_tma_chunks(g.K, kc_max, nstage);
    const size_t smem = closure_tma_smem(g.K, pad);
    CUtensorMap tmA{}, tmZ{};
    const bool tma = closure_tensor_maps(g, kc_max, &tmA, &tmZ);
    LaunchScope ls(ctx, "closure_tma_f32", flops, bytes);
    GemmDesc gd = g;
    gd.wait_flag = ctx->d_wait;
    auto go = [&](auto kern) {
      smem_attr((const void*)kern, (int)kClosureTmaSmem, ctx->device);
      kern<<<(unsigned)grid, kThreads, smem, ctx->stream>>>(gd, kc_max, nstage, tmA, tmZ);
    };
    if (tma) {
      if (pad == 12) go(closure_tma_kernel<3, 3, 12, 12, true>);
      else if (pad == 24) go(closure_tma_kernel<6, 6, 24, 24, true>);
      else go(closure_tma_kernel<4, 8, 32, 32, true>);
    } else {
      if (pad == 12) go(closure_tma_kernel<3, 3, 12, 12, false>);
      else if (pad == 24) go(closure_tma_kernel<6, 6, 24, 24, false>);
      else go(closure_tma_kernel<4, 8, 32, 32, false>);
    }
    CUDA_LAUNCH_CHECK();
    return;
  }
  LaunchScope ls(ctx, sizeof(T) == 8 ? "closure_f64" : "closure_f32", flops, bytes);
  closure_kernel<T><<<grid, kThreads, 0, ctx->stream>>>(g);
  CUDA_LAUNCH_CHECK();
}

template void launch_closure<double>(ttn_ctx*, const GemmDesc&);
template void launch_closure<float>(ttn_ctx*, const GemmDesc&);

// ---- level stage on tensor cores: TF32 MMA with the 3xTF32 split ------------------------------
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi); a*b ~ hi_a*hi_b + hi_a*lo_b + lo_a*hi_b with
// float32 accumulation, which keeps ~2^-21 relative accuracy per product (plain TF32 would give
// ~2^-11). Fragments follow the m16n8k8 .row.col layout: groupID g = lane/4, t = lane%4;
// A: a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4); B: b0 (k=t, n=g), b1 (k=t+4, n=g);
// C: c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// out[r][a] = sum_b in[b][r] E[a][b]: rows r -> MMA rows (16 per warp, 128 per CTA), a -> 8-wide
// n tiles (NT of them), b -> 8-deep k steps (KS of them). The environment slice is staged in
// shared memory as Es[n][k] (row length KS*8 + 4: conflict-free fragment loads); the output
// tile goes through a padded shared tile for coalesced stores.
template <int NT, int KS>
__global__ void __launch_bounds__(kThreads) level_tc_kernel(GemmDesc g, int rtiles) {
  constexpr int NP = NT * 8, KP = KS * 8, LDE = KP + 4, LDO = NP + 1, ROWS = 128;
  __shared__ __align__(16) float Es[NP * LDE];
  __shared__ float Os[ROWS * LDO];
  const long long bid = blockIdx.x;
  const int rt = (int)(bid % rtiles);
  const long long rest = bid / rtiles;
  const int sub = (int)(rest % g.st.n_sub);
  const int pair = (int)(rest / g.st.n_sub);
  const float* Abase = operand_base<float>(g.A, pair, g.pair_bra, g.pair_ket);
  const float* Bbase = operand_base<float>(g.B, pair, g.pair_bra, g.pair_ket);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int r0 = rt * ROWS;
  const int rw = r0 + warp * 16;                  // first row of this warp
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (int seg = g.st.seg_ptr[sub]; seg < g.st.seg_ptr[sub + 1]; ++seg) {
    const float* Ab = Abase + g.st.seg_a[seg];
    const float* Bb = Bbase + g.st.seg_b[seg];
    __syncthreads();
    for (int i = threadIdx.x; i < NP * KP; i += kThreads) {
      const int n = i / KP, k = i % KP;
      Es[n * LDE + k] = (n < g.N && k < g.K) ? Bb[(long long)n * g.b_sn + (long long)k * g.b_sk]
                                             : 0.f;
    }
    __syncthreads();
    const bool r_lo = rw + gq < g.M, r_hi = rw + gq + 8 < g.M;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * 8 + tq, k1 = k0 + 4;
      const float x0 = (r_lo && k0 < g.K) ? Ab[(long long)k0 * g.a_sk + rw + gq] : 0.f;
      const float x1 = (r_hi && k0 < g.K) ? Ab[(long long)k0 * g.a_sk + rw + gq + 8] : 0.f;
      const float x2 = (r_lo && k1 < g.K) ? Ab[(long long)k1 * g.a_sk + rw + gq] : 0.f;
      const float x3 = (r_hi && k1 < g.K) ? Ab[(long long)k1 * g.a_sk + rw + gq + 8] : 0.f;
      uint32_t ah[4], al[4];
      split_tf32(x0, ah[0], al[0]);
      split_tf32(x1, ah[1], al[1]);
      split_tf32(x2, ah[2], al[2]);
      split_tf32(x3, ah[3], al[3]);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const float* e = Es + (j * 8 + gq) * LDE + ks * 8 + tq;
        uint32_t bh[2], bl[2];
        split_tf32(e[0], bh[0], bl[0]);
        split_tf32(e[4], bh[1], bl[1]);
        mma_tf32(acc[j], al, bh);
        mma_tf32(acc[j], ah, bl);
        mma_tf32(acc[j], ah, bh);
      }
    }
  }
  // stage and store
  const int lr = warp * 16 + gq;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    Os[lr * LDO + j * 8 + 2 * tq] = acc[j][0];
    Os[lr * LDO + j * 8 + 2 * tq + 1] = acc[j][1];
    Os[(lr + 8) * LDO + j * 8 + 2 * tq] = acc[j][2];
    Os[(lr + 8) * LDO + j * 8 + 2 * tq + 1] = acc[j][3];
  }
  __syncthreads();
  long long cidx = 0;
  if (g.c_mode == MODE_PAIR) cidx = pair;
  else if (g.c_mode == MODE_BRA) cidx = g.pair_bra[pair];
  else if (g.c_mode == MODE_KET) cidx = g.pair_ket[pair];
  float* dst = static_cast<float*>(g.C) + cidx * g.c_pstride + g.st.sub_c[sub] + (long long)r0 * g.c_sm;
  const int nrow = min(ROWS, g.M - r0);
  for (int i = threadIdx.x; i < nrow * g.N; i += kThreads)
    dst[i] = Os[(i / g.N) * LDO + (i % g.N)];
}

bool level_tc_ok(const GemmDesc& g) { return level_shape_ok(g) && g.N <= 32 && g.K <= 64; }

void launch_level_tc(ttn_ctx* ctx, const GemmDesc& g) {
  if (g.n_pairs <= 0 || g.st.n_sub <= 0 || g.M <= 0 || g.N <= 0) return;
  TTN_REQUIRE(level_tc_ok(g), "tensor-core level kernel: unsupported shape");
  check_bounds(g, sizeof(float));
  const int rtiles = (g.M + 127) / 128;
  const long long grid = (long long)rtiles * g.st.n_sub * g.n_pairs;
  TTN_REQUIRE(grid <= 0x7fffffffLL, "level grid too large");
  long long nseg = 0;
  for (int q = 0; q < g.st.n_sub; ++q) nseg += g.hst->seg_ptr[q + 1] - g.hst->seg_ptr[q];
  const double flops = 2.0 * g.M * g.N * (double)g.K * nseg * g.n_pairs;
  LaunchScope ls(ctx, "level_tf32x3", flops, algorithmic_bytes(g, sizeof(float)));
  const int nt = (g.N + 7) / 8, ks = (g.K + 7) / 8;
  cudaStream_t s = ctx->stream;
#define TTN_LTC(NTv, KSv) \
  if (nt == NTv && ks == KSv) { level_tc_kernel<NTv, KSv><<<grid, kThreads, 0, s>>>(g, rtiles); }
#define TTN_LTC_K(NTv) TTN_LTC(NTv, 1) else TTN_LTC(NTv, 2) else TTN_LTC(NTv, 3) else \
  TTN_LTC(NTv, 4) else TTN_LTC(NTv, 5) else TTN_LTC(NTv, 6) else TTN_LTC(NTv, 7) else TTN_LTC(NTv, 8)
  TTN_LTC_K(1) else TTN_LTC_K(2) else TTN_LTC_K(3) else TTN_LTC_K(4)
#undef TTN_LTC_K
#undef TTN_LTC
  CUDA_LAUNCH_CHECK();
}

template void launch_level<double>(ttn_ctx*, const GemmDesc&);
template void launch_level<float>(ttn_ctx*, const GemmDesc&);

template void launch_op_stage<double>(ttn_ctx*, const OpStageDesc&);
template void launch_op_stage<float>(ttn_ctx*, const OpStageDesc&);

template void launch_gemm<double>(ttn_ctx*, const GemmDesc&);
template void launch_gemm<float>(ttn_ctx*, const GemmDesc&);
template void launch_permute<double>(ttn_ctx*, const double*, double*, long long, int,
                                     const int*, const int*);
template void launch_permute<float>(ttn_ctx*, const float*, float*, long long, int, const int*,
                                    const int*);
template void launch_pair_dot<double>(ttn_ctx*, const double*, long long, const double*,
                                      long long, long long, int, const int*, double*, int,
                                      long long, long long);
template void launch_pair_dot<float>(ttn_ctx*, const float*, long long, const float*, long long,
                                     long long, int, const int*, double*, int, long long,
                                     long long);
template void launch_shift_axpy<double>(ttn_ctx*, double*, const double*, const double*, int,
                                        long long);
template void launch_shift_axpy<float>(ttn_ctx*, float*, const float*, const double*, int,
                                       long long);
