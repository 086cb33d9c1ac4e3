// Internal declarations of libttn (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ttn.h"

// ------------------------------------------------------------------------------------------------
// errors: internal code throws TtnError; every extern "C" entry point converts it to a status.
// ------------------------------------------------------------------------------------------------
struct TtnError {
  ttn_status st;
  std::string msg;
};

std::string ttn_fmt(const char* f, ...);
#define TTN_FAIL(st, ...) throw TtnError{(st), ttn_fmt(__VA_ARGS__)}
#define TTN_REQUIRE(cond, ...) \
  do {                         \
    if (!(cond)) TTN_FAIL(TTN_EINVAL, __VA_ARGS__); \
  } while (0)
#define CUDA_CHECK(x)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      TTN_FAIL(e_ == cudaErrorMemoryAllocation ? TTN_ENOMEM : TTN_ECUDA, "%s: %s (%s:%d)", \
               #x, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
  } while (0)
#define CUDA_LAUNCH_CHECK() CUDA_CHECK(cudaGetLastError())

// Values of the context's wait flag: a bulk-copy kernel gave up waiting (copies may still have
// been landing when its CTA left), or the bounded-wait self-test ran out (nothing in flight).
enum : unsigned { TTN_WAIT_FLAG_COPY = 1u, TTN_WAIT_FLAG_SELFTEST = 2u, TTN_WAIT_FLAG_MMA = 3u };

// ------------------------------------------------------------------------------------------------
// tree
// ------------------------------------------------------------------------------------------------
struct TreeInfo {
  int n = 0, root = -1;
  std::vector<int> parent, phys;            // phys = 0 for auxiliary nodes
  std::vector<std::vector<int>> children;   // increasing index order
  std::vector<std::vector<int>> legs;       // neighbour of each leg: parent first, then children
  std::vector<int> pre, post;               // depth-first pre-/post-order from the root
  int d(int i) const { return phys[i] > 0 ? phys[i] : 1; }
  int nlegs(int i) const { return (int)legs[i].size(); }
  int leg_to(int i, int nb) const {
    for (int m = 0; m < nlegs(i); ++m)
      if (legs[i][m] == nb) return m;
    return -1;
  }
  std::vector<int> path(int u, int v) const;   // nodes from u to v inclusive
  bool same_shape(const TreeInfo& o) const { return parent == o.parent && phys == o.phys; }
};

TreeInfo make_tree(int n, const int* parent, const int* phys);

struct ttn_ctx;
struct ttn_tree {
  ttn_ctx* ctx = nullptr;
  TreeInfo info;
};

// ------------------------------------------------------------------------------------------------
// device memory: stream-ordered allocations from the device's default pool
// ------------------------------------------------------------------------------------------------
struct ttn_ctx;
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = 0;
  DevBuf() = default;
  DevBuf(size_t n, cudaStream_t st);
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept;
  ~DevBuf();
  void reset();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Launch statistics: when profiling is on, each launch is bracketed by CUDA events on the
// context stream and attributed to a kernel name with its algorithmic flops and bytes.
struct LaunchRecord {
  int name;
  cudaEvent_t start, stop;
  double flops, bytes;
};
struct ttn_ctx {
  int device = 0;
  int sm_count = 0;   // streaming multiprocessors of the device (persistent grids)
  cudaStream_t stream = 0;
  bool own_stream = false;
  std::string last_error;
  long long launches = 0;
  bool profiling = false;
  std::vector<std::string> prof_names;
  std::vector<LaunchRecord> prof;
  std::vector<cudaEvent_t> event_pool;
  double flops_total = 0.0;      // algorithmic flops of every GEMM launched (always counted)
  bool tf32x3 = false;           // float32 calls route level stages to tensor cores
  bool tc05 = false;             // ... and those stages to the tcgen05 kernels
  bool capturing = false;        // a CUDA graph is being captured on the stream (no events)
  // Set (host-mapped) by a kernel whose bounded wait on a barrier gave up (TTN_WAIT_FLAG_*);
  // read and cleared by the next entry point, which then returns TTN_ETIMEOUT.
  unsigned* h_wait = nullptr;
  unsigned* d_wait = nullptr;
  // Iteration clock of the last ttn_lobpcg / ttn_inverse_iteration call: an event at its start
  // and one after each iteration (index 0: the initial Rayleigh quotients), on the stream.
  std::vector<cudaEvent_t> iter_ev;
  int iter_marks = 0;
  // Per-launch log (kernel name, algorithmic flops and bytes, one line per launch issued outside
  // graph capture), opened when the environment variable TTN_LAUNCH_LOG names a file; lets a
  // counter capture of single launches be matched with the work those launches did.
  FILE* launch_log = nullptr;
};

// Records the iteration clock's start (mark 0 .. ) on the context stream.
// Prepares ttn_rayleigh_ritz_noalloc on the current device (see solvers.cu).
void rr_noalloc_prepare(int device);
void iter_clock_start(ttn_ctx* ctx);
void iter_clock_mark(ttn_ctx* ctx);

// Sets ctx->tf32x3 / ctx->tc05 for the duration of one entry-point call.
struct PrecisionScope {
  ttn_ctx* ctx;
  bool saved, saved_tc05;
  PrecisionScope(ttn_ctx* c, int prec) : ctx(c), saved(c->tf32x3), saved_tc05(c->tc05) {
    ctx->tf32x3 = prec == TTN_TF32X3 || prec == TTN_TF32X3_TC05;
    ctx->tc05 = prec == TTN_TF32X3_TC05;
  }
  ~PrecisionScope() {
    ctx->tf32x3 = saved;
    ctx->tc05 = saved_tc05;
  }
};
inline bool valid_precision(int prec) {
  return prec == TTN_FP64 || prec == TTN_FP32 || prec == TTN_TF32X3 || prec == TTN_TF32X3_TC05;
}
// float64 for TTN_FP64, float32 otherwise
inline bool is_fp64(int prec) { return prec == TTN_FP64; }

// RAII helper: records the launch's events (if profiling) and counts it.
struct LaunchScope {
  ttn_ctx* ctx;
  int idx = -1;
  LaunchScope(ttn_ctx* c, const char* name, double flops, double bytes);
  ~LaunchScope();
};

// RAII helper for a driver phase ("phase:<name>"): events only, no launch counted.
struct PhaseScope {
  ttn_ctx* ctx;
  int idx = -1;
  PhaseScope(ttn_ctx* c, const char* name);
  ~PhaseScope();
};

// ------------------------------------------------------------------------------------------------
// TTNO
// ------------------------------------------------------------------------------------------------
struct TtnoEntry {
  int w[TTN_MAX_LEGS];
  int op;        // index into the op table
  double coef;
};

// Symbolic plan of one node contraction with one open leg (or none): the prefix tries over
// the contracted legs and the per-output-slot groups with their combined local operators.
struct NodePlan {
  int node = -1, open = -1;
  DevBuf d_slot_ptr, d_grp_prefix;                     // device copies for the operator stage
  std::vector<int> C;                                  // contracted legs in order
  std::vector<std::vector<std::pair<int, int>>> level; // level[l]: (parent prefix, w) per prefix
  int n_slots = 1;
  std::vector<int> grp_prefix;                         // per group (sorted by slot)
  std::vector<int> slot_ptr;                           // CSR over slots
  std::vector<double> ocomb;                           // per group: d x d  sum_e c_e O_e
  DevBuf d_ocomb64, d_ocomb32;
  // Operator-first variant for nodes without a physical leg (d = 1) and m >= 1 contracted
  // legs: the TTNO is folded into the last contracted leg's environment,
  //   Et[G][a][b] = sum_{entries e in G} c_e E_Cm[w_Cm(e)][a][b],  G = (prefix_{m-1}, slot),
  // and Z[slot] = sum_{G in slot} T_{m-1}[prefix(G)] x_Cm Et[G] is one segmented level stage.
  bool fused = false;
  std::vector<int> fG_prefix;        // per G: prefix index at level m-1 (0 if m == 1)
  std::vector<int> fG_slot_ptr;      // CSR over slots
  std::vector<int> fG_term_ptr;      // CSR over G: terms
  std::vector<int> fT_w;             // per term: w of the last contracted leg
  std::vector<double> fT_coef;       // per term: coefficient (times the 1 x 1 operator)
  DevBuf d_fG_term_ptr, d_fT_w, d_fT_coef64, d_fT_coef32;
};

// Item tables of one GEMM stage: per item ("sub") the C offset and a CSR list of segments,
// each with its own A and B offsets (device copy for the kernel, host copy for bounds checks).
// Level stages also carry "A groups": lists of single-segment items that read the same A slice
// (children of one prefix in the TTNO trie), so one staged A tile serves all of them.
struct StageDev {
  int n_sub = 0;
  const long long* sub_c = nullptr;
  const int* seg_ptr = nullptr;
  const long long* seg_a = nullptr;
  const long long* seg_b = nullptr;
  int n_grp = 0;                    // 0: no A groups (some item has several segments)
  const int* grp_ptr = nullptr;     // CSR over grp_sub, n_grp + 1 entries
  const int* grp_sub = nullptr;
  const long long* grp_a = nullptr;   // per group: the shared A offset
  const long long* grp_b = nullptr;   // per member (aligned with grp_sub): its B offset
  const long long* grp_c = nullptr;   // per member: its C offset
};
struct StageHost {
  std::vector<long long> sub_c, seg_a, seg_b;
  std::vector<int> seg_ptr{0};
  std::vector<int> grp_ptr{0}, grp_sub;
  std::vector<long long> grp_a, grp_b, grp_c;
  // facts the launchers need on every launch, computed once when the tables are built
  long long n_ua = -1, n_ub = -1;   // distinct A / B offsets (-1: not computed)
  long long n_seg = 0;              // segments over all items
  bool single = true;               // every item has exactly one segment
  bool a4 = true, b4 = true;        // every A / B offset a multiple of 4 elements
  bool c2 = true;                   // every C offset even
  bool c4 = true;                   // every C offset a multiple of 4 elements
  int grp_max = 0;                  // largest A group
  void finalize();
};
struct DevTables {
  DevBuf buf;   // all item tables of one (plan, dims) in one allocation
  std::vector<StageDev> stages;
  std::vector<StageHost> host;
};

struct ttn_ttno {
  ttn_ctx* ctx = nullptr;
  TreeInfo tree;
  std::vector<int> wbond;
  std::vector<int> op_node;
  std::vector<long long> op_off;
  std::vector<double> op_data;
  std::vector<std::vector<TtnoEntry>> entries;
  // Per edge (child node): numerical rank of the sum-of-products coefficient matrix across the
  // edge, the smallest bond of any exact TTNO of H there (-1 where unknown, 1 at the root).
  std::vector<int> rank_bound;
  std::map<long long, NodePlan> plans;
  std::map<std::vector<long long>, DevTables> tables;
  int wdim(int node, int leg) const {
    int nb = tree.legs[node][leg];
    return tree.parent[node] == nb ? wbond[node] : wbond[nb];
  }
};

NodePlan& get_plan(ttn_ttno* H, int node, int open);
ttn_ttno* identity_ttno(ttn_ctx* ctx, const TreeInfo& tree);

// ------------------------------------------------------------------------------------------------
// blocks and environments
// ------------------------------------------------------------------------------------------------
struct ttn_block {
  ttn_ctx* ctx = nullptr;
  TreeInfo tree;
  int n_states = 0;
  std::vector<int> bond;                      // per node (edge to parent)
  std::vector<std::vector<int>> dims;         // per node: leg dims then physical (1 for aux)
  std::vector<long long> size, off;           // per node: tensor size, slab offset
  long long total = 0;
  DevBuf d64;
  mutable DevBuf d32;
  mutable bool f32_valid = false;
  int bdim(int node, int leg) const {
    int nb = tree.legs[node][leg];
    return tree.parent[node] == nb ? bond[node] : bond[nb];
  }
  double* node64(int t) const { return d64.as<double>() + off[t]; }
  const float* node32(int t) const;           // refreshes the float mirror if stale
  void touch() { f32_valid = false; }
};

struct ttn_envs {
  ttn_ctx* ctx = nullptr;
  TreeInfo tree;
  int n_pairs = 0;
  int prec = TTN_FP64;
  bool has_up = false, has_down = false;
  std::vector<int> Dw, Da, Db;                // per edge (child node)
  std::vector<DevBuf> up, down;               // per edge: [pair][w][a][b]
  std::vector<int> pair_bra, pair_ket;
  const ttn_ttno* H = nullptr;
  long long esize(int t) const { return (long long)Dw[t] * Da[t] * Db[t]; }
};

// ------------------------------------------------------------------------------------------------
// kernels (kernels.cu)
// ------------------------------------------------------------------------------------------------
enum { MODE_PAIR = 0, MODE_BRA = 1, MODE_KET = 2, MODE_CONST = 3 };

struct GemmOperand {
  const void* base;
  int mode;
  long long pstride;
};

struct GemmDesc {
  int M, N, K;
  long long a_sm, a_sk, b_sn, b_sk, c_sm, c_sn;
  GemmOperand A, B;
  void* C;
  int c_mode;
  long long c_pstride;
  int n_pairs;
  const int* pair_bra;
  const int* pair_ket;
  StageDev st;
  // host-side launch validation (never read on the device)
  const StageHost* hst;
  long long a_len, b_len, c_len;   // elements addressable from each base pointer
  int max_bra, max_ket;            // largest state index in pair_bra / pair_ket
  unsigned* wait_flag;             // device view of ttn_ctx::h_wait (set by the launcher)
  // Which operands count as algorithmic bytes: node tensors (read once per distinct state),
  // environments and results; intermediates of the contraction chain do not count.
  bool alg_a, alg_b, alg_c;
};

// A list of (bra, ket) pairs on the device plus the host facts the bounds checks need.
struct PairSet {
  int P = 0;
  const int* d_pb = nullptr;
  const int* d_pk = nullptr;
  int max_bra = 0, max_ket = 0;
};

template <class T> void launch_gemm(ttn_ctx* ctx, const GemmDesc& g);
// Et[pair][G] = sum_{t in G} coef_t E[pair][w_t] (operator-first fold of a d = 1 node); the
// da x db slices [a][b] of E are written transposed ([b][a]) into Et.
template <class T>
void launch_combine_env(ttn_ctx* ctx, const T* E, long long e_pstride, int da, int db, T* Et,
                        int n_pairs, int nG, const int* term_ptr, const int* term_w,
                        const T* term_coef, int max_w);
// Specialised level-stage GEMM (a_sm = 1, N, K <= 64; items sum over their segments).
bool level_shape_ok(const GemmDesc& g);
// Largest A-group size the bulk-copy level kernel stages for an (M, N, K) float level stage
// (0 when that kernel does not take the shape).
int level_group_cap(int M, int N, int K);
template <class T> void launch_level(ttn_ctx* ctx, const GemmDesc& g);
// Tensor-core (TF32 MMA, 3xTF32 split) level stage for float data, N <= 32, K <= 64.
bool level_tc_ok(const GemmDesc& g);
void launch_level_tc(ttn_ctx* ctx, const GemmDesc& g);
// Specialised closure GEMM (one segment per item, a_sk = b_sk = 1, M, N <= 32).
bool closure_shape_ok(const GemmDesc& g);
template <class T> void launch_closure(ttn_ctx* ctx, const GemmDesc& g);

// Operator stage of a node contraction (see engine.cu):
//   Z[pair][slot][r][p] = sum_{g in slot} sum_q Tm[pair][prefix_g][q][r] * O_g[p][q]
struct OpStageDesc {
  int d, rows, n_slots, n_groups;
  long long tsize;          // d * rows: one prefix slice of Tm
  GemmOperand A;            // Tm base (pair- or ket-indexed)
  const int* slot_ptr;      // [n_slots + 1]
  const int* grp_prefix;    // [n_groups]
  const void* ops;          // [n_groups][d][d]
  void* Z;
  long long z_pstride;      // n_slots * d * rows
  int n_pairs;
  const int* pair_bra;
  const int* pair_ket;
  // host-side validation
  long long a_len, z_len;
  int max_ket, max_prefix;
  int n_unique_prefix;      // distinct T_m slices read
  bool alg_in, alg_out;     // input is a node tensor / output is the contraction's result
};
template <class T> void launch_op_stage(ttn_ctx* ctx, const OpStageDesc& o);
template <class T>
void launch_permute(ttn_ctx* ctx, const T* in, T* out, long long batch, int nd, const int* dims,
                    const int* perm);
template <class T>
void launch_pair_dot(ttn_ctx* ctx, const T* bra, long long bra_stride, const T* Z,
                     long long z_stride, long long n, int n_pairs, const int* pair_bra,
                     double* out, int max_bra, long long bra_len, long long z_len);
template <class T>
void launch_shift_axpy(ttn_ctx* ctx, T* y, const T* x, const double* shift, int n_states,
                       long long size);
void launch_to_f32(ttn_ctx* ctx, const double* in, float* out, long long n);
void launch_to_f64(ttn_ctx* ctx, const float* in, double* out, long long n);
void launch_scatter_gram(ttn_ctx* ctx, const double* g, int n_pairs, const int* pb,
                         const int* pk, int symmetric, double* out, int ld);
// dst[j][:] = src[d_idx[j]][:] for j < n_rows (rows of `size` doubles; d_idx on the device).
void launch_gather_rows(ttn_ctx* ctx, double* dst, const double* src, const int* d_idx,
                        int n_rows, long long size);
// Counts the non-finite entries of rows x cols (leading dimension ld) into *d_count (device).
void launch_count_nonfinite(ttn_ctx* ctx, const double* a, int rows, int cols, int ld,
                            unsigned* d_count);
// One CTA whose barrier wait cannot complete waits for budget_ns and raises the wait flag.
void launch_wait_selftest(ttn_ctx* ctx, unsigned long long budget_ns);

// ------------------------------------------------------------------------------------------------
// engine (engine.cu)
// ------------------------------------------------------------------------------------------------
enum { OUT_ENV = 0, OUT_SCALAR = 1, OUT_LOCAL = 2 };

// Contract node t (see engine.cu). `ket` supplies the ket bond dimensions and, unless
// ket_ptr is given, the ket tensors; ket_ptr (ket_n states of the node's size, contiguous)
// replaces them, e.g. with Krylov vectors.
template <class T>
void node_op(ttn_ctx* ctx, ttn_ttno* H, int t, int open, const ttn_block* bra,
             const ttn_block* ket, const PairSet& ps, const std::vector<const T*>& env,
             const std::vector<int>& env_da, void* out, long long out_len, int out_kind,
             const T* ket_ptr = nullptr, int ket_n = 0);

template <class T>
void envs_compute(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                  const PairSet& ps, int direction, std::vector<DevBuf>& up,
                  std::vector<DevBuf>& down);

template <class T> const T* block_node(const ttn_block* b, int t);
