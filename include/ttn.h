/*
 * libttn — GB300 (sm_103a) hot path of the tree-tensor-network vibrational eigensolver.
 *
 * The library evaluates, on one GPU, the contractions that dominate LOBPCG and inverse
 * iteration on tree tensor network states (TTNS, Eq. ttns) with a Hamiltonian given as a tree
 * tensor network operator (TTNO, Eq. ttno) built from a sum of products (Eq. sum_of_tp):
 * environment (cache) updates, the local effective-Hamiltonian apply, block Gram matrices,
 * the exact TTNO x TTNS product, variational fitting, ALS solves and block LOBPCG.
 *
 * Conventions shared by every call
 *   - All values are real double precision on the host side of the ABI (the vibrational
 *     Hamiltonians are real symmetric; complex conjugation of bra tensors is the identity).
 *   - Tree: parent[i] = -1 for the root; phys_dim[i] = 0 marks an auxiliary node (no physical
 *     leg). Children of a node are ordered by increasing node index.
 *   - Node tensor layout (row-major): (parent leg, children legs in index order, physical leg).
 *     The root has no parent leg, an auxiliary node no physical leg.
 *   - Bonds: bond_dims[i] is the dimension of edge (i, parent(i)); bond_dims[root] is ignored.
 *   - Environment layout for one (bra, ket) pair and one edge: E[w][a][b] (TTNO bond w, bra
 *     bond a, ket bond b), row-major. "up" environments contract the subtree below the edge,
 *     "down" environments everything outside it.
 *   - Handles are created and destroyed by the library. Host arrays passed in are owned by the
 *     caller and only read during the call. Device memory behind a handle is owned by it.
 *   - Every call returns a ttn_status; no exception crosses the ABI. On failure, the context's
 *     ttn_last_error() holds a one-line message. TTN_ENOTCONV is informational: results are
 *     written.
 *   - Work is issued on the context's stream. Calls that return host data synchronise it.
 *   - Results are deterministic for identical inputs (fixed reduction order).
 */
#ifndef TTN_H
#define TTN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TTN_OK = 0,
  TTN_EINVAL = 1,        /* bad argument (size, index, tree shape, NULL pointer) */
  TTN_ENOMEM = 2,        /* device or host allocation failed */
  TTN_ECUDA = 3,         /* a CUDA runtime call failed */
  TTN_ENONFINITE = 4,    /* a NaN/Inf appeared in a result that is checked */
  TTN_ENOTCONV = 5,      /* an iteration hit its cap before its tolerance (results written) */
  TTN_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  TTN_EUNSUPPORTED = 7   /* valid request outside what this build implements */
} ttn_status;

typedef enum {
  TTN_FP64 = 0,   /* every contraction in float64 */
  TTN_FP32 = 1,   /* node contractions in float32 with float32 accumulation; Gram closure,
                     Lanczos/MINRES scalars and Rayleigh-Ritz in float64 */
  TTN_TF32X3 = 2, /* as TTN_FP32, but the level stages of the node contractions run on the
                     tensor cores as TF32 products with the 3xTF32 split (x = hi + lo, three
                     products per term) and float32 accumulation (mma.sync kernels) */
  TTN_TF32X3_TC05 = 3 /* as TTN_TF32X3, with the level stages on the fifth-generation tensor
                         cores: tcgen05.mma kind::tf32 from shared-memory operand descriptors
                         into float32 accumulators in tensor memory */
} ttn_precision;

#define TTN_MAX_LEGS 8   /* stride of per-entry w-tuples in the TTNO entry arrays */

typedef struct ttn_ctx ttn_ctx;
typedef struct ttn_tree ttn_tree;
typedef struct ttn_ttno ttn_ttno;
typedef struct ttn_block ttn_block;
typedef struct ttn_envs ttn_envs;

/* ---- context ---------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to issue work on,
 * or NULL for a stream owned by the context. device = -1 creates a host-only context that
 * can create trees and build, import and export TTNOs, and nothing else (no GPU needed).
 * On a device, creation also prepares ttn_rayleigh_ritz_noalloc there (once per device). */
ttn_status ttn_create(ttn_ctx** out, int device, void* cuda_stream);
void ttn_destroy(ttn_ctx* ctx);
/* Message of the last failing call on this context ("" if none). Valid until the next call. */
const char* ttn_last_error(const ttn_ctx* ctx);
/* Block the host until all work issued on the context's stream has finished. */
ttn_status ttn_synchronize(ttn_ctx* ctx);
/* Device time (CUDA events on the context's stream) from the start of the last ttn_lobpcg or
 * ttn_inverse_iteration call on this context to the end of each of its iterations: ms[0] after
 * the initial Rayleigh quotients, ms[i] after iteration i. Writes at most max_n values and
 * returns how many the call recorded (0 if none, -1 on a CUDA error). */
int ttn_iteration_times(ttn_ctx* ctx, double* ms, int max_n);
/* Number of kernels this context has launched so far (for launch accounting). */
long long ttn_launch_count(const ttn_ctx* ctx);
/* Algorithmic flops of every contraction GEMM launched so far: 2*M*N*K per item and segment
 * of the block-sparse contraction (no padding, no zero TTNO blocks). */
double ttn_flop_count(const ttn_ctx* ctx);
/* Turn per-launch timing on (1) or off (0) and clear the records. While on, every launch is
 * bracketed by CUDA events recorded on the context's stream. */
ttn_status ttn_profile_enable(ttn_ctx* ctx, int on);
/* Per-kernel totals since the last ttn_profile_enable: kernel name (64 chars each, NUL
 * terminated), launches, summed event time in ms, algorithmic flops and bytes. Arrays hold
 * max_kernels entries; *n_kernels receives the number of distinct kernels (may exceed it). */
ttn_status ttn_profile_get(ttn_ctx* ctx, int max_kernels, char* names, long long* launches,
                           double* ms, double* flops, double* bytes, int* n_kernels);

/* ---- failure-path checks (no counterpart in the paper) ------------------------------------ */

/* Runs one device block whose barrier wait can never complete (it announces a transfer that no
 * copy delivers; nothing is in flight) with a wait budget of budget_ms (0.001 .. 1000 ms) and
 * returns what every entry point returns after such a wait gives up: TTN_ETIMEOUT, with a
 * message. The context stays usable afterwards. This exercises, without any GPU fault, the
 * bounded waits that the bulk-copy kernels use (2 s budget); after a real TTN_ETIMEOUT from
 * those kernels, copies may still have been in flight, and the context must be destroyed. */
ttn_status ttn_selftest_bounded_wait(ttn_ctx* ctx, double budget_ms);
/* Process-wide allocation-failure injection: after `after` further device allocations of the
 * library succeed, the next one fails as an out-of-memory allocation would (the call that made
 * it returns TTN_ENOMEM) and injection switches itself off. after < 0 switches it off. */
void ttn_fault_inject_alloc(long long after);

/* ---- tree (Sec. II.A.2, Eq. ttns; Appendix B trees) -------------------------------------- */

/* parent[n_nodes]: -1 exactly once (the root), otherwise a node index, no cycles.
 * phys_dim[n_nodes]: local basis size d >= 1, or 0 for an auxiliary node. At most
 * TTN_MAX_LEGS-1 children per node. */
ttn_status ttn_tree_create(ttn_ctx* ctx, int n_nodes, const int* parent, const int* phys_dim,
                           ttn_tree** out);
void ttn_tree_destroy(ttn_tree* tree);

/* ---- TTNO (Sec. II.A.3, Eq. sum_of_tp, Eq. ttno) ----------------------------------------- */

/* Build a TTNO of H = sum_t coeff[t] prod_{o in term t} op_o from a sum of products.
 *   op_site[n_ops]      node carrying operator o (a node with a physical leg);
 *   op_offset[n_ops+1]  op_data[op_offset[o] .. op_offset[o+1]) is op o, d x d row-major
 *                       with d = phys_dim[op_site[o]];
 *   coeff[n_terms], term_offset[n_terms+1], term_op_ids[term_offset[n_terms]]: term t is
 *                       coeff[t] times the product of ops term_op_ids[term_offset[t]..);
 *                       at most one op per node within a term.
 *   tol                 relative tolerance for treating two rows/columns of an edge's
 *                       coefficient matrix as proportional (e.g. 1e-12).
 * Construction: leaves-to-root sweep over the edges; on each edge the terms split into a
 * subtree part and a rest part, proportional rows/columns of the bipartite coefficient matrix
 * are merged, and a minimum vertex cover of the merged bipartite graph (Koenig's theorem)
 * chooses the bond channels. Each TTNO entry stays one local operator times a coefficient.
 * bond_dims_out[n_nodes] (may be NULL) receives the TTNO bond of each edge (1 at the root). */
ttn_status ttn_build_ttno(ttn_ctx* ctx, const ttn_tree* tree, int n_ops, const int* op_site,
                          const long long* op_offset, const double* op_data, int n_terms,
                          const double* coeff, const int* term_offset, const int* term_op_ids,
                          double tol, ttn_ttno** out, int* bond_dims_out);

/* Lower bound on the operator bond of each edge (the TTNO paragraph of Sec. II.A.3): rank_out[i]
 * for the edge (i, parent(i)) is the numerical rank (pivoted QR, float64, relative tolerance
 * 1e-12) of the matrix of term coefficients indexed by the term's operator string on the subtree
 * of i and its string on the rest of the tree, the smallest bond any exact TTNO of H can have
 * there when distinct operator strings are linearly independent. 1 at the root; -1 on every
 * edge of a TTNO made by ttn_ttno_create (no terms known). Compare with bond_dims_out of
 * ttn_build_ttno. */
ttn_status ttn_ttno_rank_bounds(const ttn_ttno* H, int* rank_out);

/* Create a TTNO from explicit entries (no arithmetic): operator bonds wbond[n_nodes] (root
 * ignored), an op table as in ttn_build_ttno, and n_entries entries with entry_node[e],
 * w-tuple entry_w[e*TTN_MAX_LEGS + m] for the node's legs m in tensor order, op index
 * entry_op[e] and coefficient entry_coef[e]. W[w-tuple][p][q] += coef * op[p][q]. */
ttn_status ttn_ttno_create(ttn_ctx* ctx, const ttn_tree* tree, const int* wbond, int n_ops,
                           const int* op_site, const long long* op_offset,
                           const double* op_data, int n_entries, const int* entry_node,
                           const int* entry_w, const int* entry_op, const double* entry_coef,
                           ttn_ttno** out);
/* Sizes of a TTNO: wbond_out[n_nodes] (may be NULL), total entries, total op-table doubles. */
ttn_status ttn_ttno_info(const ttn_ttno* H, int* wbond_out, int* n_entries_out,
                         long long* n_op_doubles_out);
/* Export the entries (arrays sized from ttn_ttno_info): entry_node, entry_w (TTN_MAX_LEGS per
 * entry), entry_coef, and each entry's own operator at op_data[op_offset[e] ..). */
ttn_status ttn_ttno_get_entries(const ttn_ttno* H, int* entry_node, int* entry_w,
                                double* entry_coef, long long* op_offset, double* op_data);
void ttn_ttno_destroy(ttn_ttno* H);

/* ---- block of TTNS (Sec. II.A.2; the LOBPCG block of Alg. 2) ------------------------------ */

/* n_states states on `tree` with bonds bond_dims[n_nodes]; device-resident, zero-initialised.
 * Node t of all states is stored contiguously as [state][tensor]. */
ttn_status ttn_block_create(ttn_ctx* ctx, const ttn_tree* tree, int n_states,
                            const int* bond_dims, ttn_block** out);
void ttn_block_destroy(ttn_block* b);
/* Copy node `node` of state `state` from/to the host (n = tensor size). state = -1 means all
 * states of that node at once (n = n_states * size, state-major). */
ttn_status ttn_block_set(ttn_block* b, int state, int node, const double* host, long long n);
ttn_status ttn_block_get(const ttn_block* b, int state, int node, double* host, long long n);
/* Tensor size of `node` and the device address of its [state][tensor] slab. */
ttn_status ttn_block_node_info(const ttn_block* b, int node, long long* size,
                               double** device_ptr);
/* dst state j := src state src_states[j] for j < n (same tree and bonds, distinct blocks);
 * one gather launch per node. */
ttn_status ttn_block_copy_states(ttn_block* dst, const ttn_block* src, int n,
                                 const int* src_states);

/* ---- environments (Sec. II.C.2-3: the cached environment blocks) ------------------------- */

ttn_status ttn_envs_create(ttn_ctx* ctx, const ttn_tree* tree, ttn_envs** out);
void ttn_envs_destroy(ttn_envs* e);
/* Compute environments of <bra_i| H |ket_j> for n_pairs pairs (pair_bra/pair_ket, host) into
 * `envs` (replacing its contents). H = NULL means the identity operator (overlap
 * environments, TTNO bond 1). direction: 0 = up only, 1 = down only (needs up, computed too),
 * 2 = both. */
ttn_status ttn_env_update(ttn_ctx* ctx, const ttn_ttno* H, const ttn_block* bra,
                          const ttn_block* ket, int n_pairs, const int* pair_bra,
                          const int* pair_ket, int direction, ttn_envs* envs,
                          ttn_precision prec);
/* Read one environment E[w][a][b] of edge (node, parent(node)) for pair index `pair`;
 * direction 0 = up, 1 = down. n must equal its size. */
ttn_status ttn_envs_get(const ttn_envs* e, int node, int direction, int pair, double* host,
                        long long n);

/* ---- local effective Hamiltonian (Sec. II.C.3, Fig. als) --------------------------------- */

/* y_s[node] = (H_eff,node(s) - shift[s]) x_s[node] for every state s, where H_eff,node(s) is
 * built from `envs` pair s (computed with ttn_env_update, direction 2, usually with bra = ket
 * = the state whose environments these are). shift may be NULL (no shift). */
ttn_status ttn_heff_apply(ttn_ctx* ctx, const ttn_ttno* H, const ttn_envs* envs, int node,
                          const ttn_block* x, ttn_block* y, const double* shift,
                          ttn_precision prec);

/* ---- block Gram (Alg. 2 "construct matrices", Alg. 3 orthogonalisation) ------------------ */

/* S[k][l] = <bra_k|ket_l>, Hm[k][l] = <bra_k|H|ket_l>, row-major with leading dimension ld.
 * Either output may be NULL. When bra == ket only k <= l is contracted and mirrored.
 * out_on_device != 0: S/Hm are device pointers. */
ttn_status ttn_gram(ttn_ctx* ctx, const ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                    double* S, double* Hm, int ld, int out_on_device, ttn_precision prec);

/* ---- exact TTNO x TTNS product (Sec. II.C.1, direct contraction) ------------------------- */

/* out = H |in> for every state; new bond of edge i is wbond[i] * bond[i] with the TTNO index
 * the major one. *out is created by the call. */
ttn_status ttn_apply_block(ttn_ctx* ctx, const ttn_ttno* H, const ttn_block* in,
                           ttn_block** out, ttn_precision prec);

/* ---- successive randomized compression (Sec. II.C.1, Figs. random tensor and src) ------- */

/* *out ~ H |x> for every state of x, by SRC with sketch dimension chi (1 .. 64). The sketch is
 * the Khatri-Rao product of per-node random matrices Omega^(i) (d_i x chi), passed in `omega`:
 * for every node with a physical leg, in node order, its d_i x chi matrix row-major (auxiliary
 * nodes have none); chi * sum_i d_i doubles, owned by the caller. Leaves to root, each node's
 * local sketch (the parent edge's sketched environment, the children's residual environments,
 * the TTNO and x) is orthogonalised by QR into the new node tensor; the root is contracted
 * directly. *out is created by the call: same tree and state count as x, bond of edge i
 * min(chi, d_i * prod of its children's bonds), canonical form toward the root. With chi at
 * least the rank of the exact product on every edge the result is H|x> up to rounding.
 * Returns TTN_ENONFINITE for a non-finite omega. */
ttn_status ttn_src_apply(ttn_ctx* ctx, const ttn_ttno* H, const ttn_block* x, int chi,
                         const double* omega, ttn_block** out, ttn_precision prec);

/* ---- variational fitting (Sec. II.C.2) ---------------------------------------------------- */

/* For j < n_out: out_j ~ sum_k coeff[k*n_out + j] * O_k |in_k>, k < n_in, where input k is
 * state in_state[k] of block in[k] and O_k = ops[k] (NULL = identity). `out` holds the initial
 * guesses on entry and the fitted states (canonical form, centre at the root) on return.
 * All blocks share the tree and bonds. */
ttn_status ttn_recompress(ttn_ctx* ctx, int n_in, const double* coeff,
                          const ttn_ttno* const* ops, const ttn_block* const* in,
                          const int* in_state, ttn_block* out, int n_out, int n_sweeps,
                          ttn_precision prec);

/* ---- ALS solve (Sec. II.C.3, Eq. solve precondition) ------------------------------------- */

/* For every state s: solve (H - shift[s] I) y_s = rhs_s by ALS sweeps with MINRES local
 * solves (at most minres_max iterations, relative tolerance minres_tol). y holds the initial
 * guess on entry. Returns TTN_ENOTCONV (results written) if a local solve hit its cap. */
ttn_status ttn_als_solve(ttn_ctx* ctx, const ttn_ttno* H, const double* shift,
                         const ttn_block* rhs, ttn_block* y, int n_sweeps, int minres_max,
                         double minres_tol, ttn_precision prec);

/* ---- Rayleigh-Ritz (Alg. 2 GEVP) ---------------------------------------------------------- */

/* Smallest n solutions of Ht v = theta Mt v (m x m, row-major, host) by canonical
 * orthogonalisation of Mt (eigenvalues below eps * max dropped), on the GPU in float64.
 * theta[n], V[m x n] row-major (column j = v_j). Returns TTN_EINVAL if fewer than n
 * directions survive. */
ttn_status ttn_rayleigh_ritz(ttn_ctx* ctx, int m, const double* Ht, const double* Mt, int n,
                             double eps, double* theta, double* V);

/* ---- block inverse iteration (Alg. 3, Eq. inverse iteration update) ----------------------- */

/* n_iter iterations of block inverse iteration on the states of x (updated in place). The
 * current Rayleigh quotients are grouped by single linkage: sorted values closer than
 * cluster_gap form one block (Sec. III.B uses 5 cm^-1); cluster_gap <= 0 gives one block per
 * state (a shift per state). Each block's shift is the mean Rayleigh quotient of its states;
 * every state solves (H - shift) y = x by ALS (als_sweeps sweeps, MINRES <= minres_max,
 * relative tolerance minres_tol) and is normalised; a block of more than one state is
 * re-orthogonalised by its own Rayleigh-Ritz step and refitted (fit_sweeps). rq_hist
 * [(n_iter+1) x n] receives the values after each iteration (row 0 = initial quotients).
 * Returns TTN_ENOTCONV (results written) if a local solve hit its cap. */
ttn_status ttn_inverse_iteration(ttn_ctx* ctx, const ttn_ttno* H, ttn_block* x, int n_iter,
                                 double cluster_gap, int als_sweeps, int minres_max,
                                 double minres_tol, int fit_sweeps, ttn_precision prec,
                                 double* rq_hist);

/* ---- generalized eigenvalue problem over a block (Sec. III.B, Alg. 3 orthogonalisation) ---- */

/* Hc = ESc over all states of x: the Gram matrices <x_k|H|x_l> and <x_k|x_l> are formed, the
 * pencil is solved by canonical orthogonalisation (overlap eigenvalues below eps * max
 * dropped), and each state is replaced by its Ritz vector sum_l c_la x_l, fitted back into x's
 * bonds (fit_sweeps sweeps) and normalised. theta[n_states] (may be NULL) receives the Ritz
 * values in ascending order. This removes the residual non-orthogonality between states that
 * block inverse iteration leaves across its blocks. Returns TTN_EINVAL if fewer than n_states
 * directions survive eps. */
ttn_status ttn_block_rayleigh_ritz(ttn_ctx* ctx, const ttn_ttno* H, ttn_block* x, double eps,
                                   int fit_sweeps, ttn_precision prec, double* theta);

/* ---- Rayleigh-Ritz without device allocation --------------------------------------------- */

/* The paper has no counterpart to this call. It serves callers that may not allocate device
 * memory once they are running: a serving process that reserves its whole device budget at
 * start-up, an application whose device memory pool is frozen after initialisation, or a host
 * framework that owns the allocator and forbids allocations from libraries it calls.
 *
 * Same result as ttn_rayleigh_ritz, but Ht, Mt (m x m, row-major), theta[n] and V[m x n] are
 * DEVICE pointers owned by the caller, and the working memory is a fixed area compiled into the
 * library: about 3.7 MB of float64 per GPU, held from library load until process exit. The call
 * allocates and frees no device memory (no cudaMalloc, no pool allocation).
 *   - m may not exceed TTN_RR_NOALLOC_MAX_M; larger m returns TTN_EINVAL with a message.
 *   - ttn_create looks up the area's device address and loads the kernels this call launches
 *     (under lazy module loading a kernel's first launch would load its code and take device
 *     memory for it), once per device, so that no call, the first included, allocates.
 *   - All calls on a device share the one area and it keeps the last call's contents (every
 *     value a call reads there, it has written first). Calls that overlap on the GPU (other
 *     streams, other threads) race on it: serialise them.
 *   - The eigenvalue problems are solved by a single-CTA cyclic Jacobi of at most 40 sweeps;
 *     if either stops with sqrt(off-diagonal / total) above 1e-10 the call returns
 *     TTN_ENOTCONV (results written).
 * Other errors as for ttn_rayleigh_ritz. The call synchronises the context's stream: it reads
 * the overlap spectrum on the host half way through, and again at the end. */
#define TTN_RR_NOALLOC_MAX_M 256
ttn_status ttn_rayleigh_ritz_noalloc(ttn_ctx* ctx, int m, const double* Ht, const double* Mt,
                                     int n, double eps, double* theta, double* V);

/* ---- block LOBPCG (Alg. 2) ---------------------------------------------------------------- */

/* n_iter iterations of block LOBPCG on the states of x (updated in place). The ALS
 * preconditioner shift is (lowest current Ritz value) + shift_offset. eig_hist[(n_iter+1) x n]
 * receives the Ritz values after each iteration (row 0 = initial Rayleigh quotients). */
ttn_status ttn_lobpcg(ttn_ctx* ctx, const ttn_ttno* H, ttn_block* x, int n_iter,
                      double shift_offset, int als_sweeps, int minres_max, double minres_tol,
                      int fit_sweeps, ttn_precision prec, double* eig_hist);

#ifdef __cplusplus
}
#endif
#endif /* TTN_H */
