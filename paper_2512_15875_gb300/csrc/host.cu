// Host-side objects of libttn: trees, the TTNO builder, blocks of states, environment caches,
// and the C-ABI entry points of the contraction calls.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <set>
#include <tuple>

#include "internal.h"

std::string ttn_fmt(const char* f, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof(buf), f, ap);
  va_end(ap);
  return buf;
}

// ------------------------------------------------------------------------------------------------
// device buffers
// ------------------------------------------------------------------------------------------------
// Allocation-failure injection (ttn_fault_inject_alloc): the number of device allocations that
// still succeed before one fails; negative when off.
static std::atomic<long long> g_alloc_countdown{-1};

DevBuf::DevBuf(size_t n, cudaStream_t st) : bytes(n), s(st) {
  if (n == 0) return;
  if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) == 0) {
    g_alloc_countdown.store(-1);
    TTN_FAIL(TTN_ENOMEM, "device allocation of %zu bytes failed: injected failure", n);
  }
  cudaError_t e = cudaMallocAsync(&p, n, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    TTN_FAIL(TTN_ENOMEM, "device allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
  }
}
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    reset();
    p = o.p;
    bytes = o.bytes;
    s = o.s;
    o.p = nullptr;
    o.bytes = 0;
  }
  return *this;
}
void DevBuf::reset() {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
  bytes = 0;
}
DevBuf::~DevBuf() { reset(); }

// ------------------------------------------------------------------------------------------------
// tree
// ------------------------------------------------------------------------------------------------
std::vector<int> TreeInfo::path(int u, int v) const {
  std::vector<int> au{u}, av{v};
  while (parent[au.back()] >= 0) au.push_back(parent[au.back()]);
  while (parent[av.back()] >= 0) av.push_back(parent[av.back()]);
  std::set<int> sv(av.begin(), av.end());
  size_t iu = 0;
  while (!sv.count(au[iu])) ++iu;
  const int common = au[iu];
  std::vector<int> out(au.begin(), au.begin() + iu + 1);
  size_t iv = 0;
  while (av[iv] != common) ++iv;
  for (size_t k = iv; k-- > 0;) out.push_back(av[k]);
  return out;
}

TreeInfo make_tree(int n, const int* parent, const int* phys) {
  TTN_REQUIRE(n >= 1 && parent && phys, "tree: need n_nodes >= 1 and non-NULL arrays");
  TreeInfo t;
  t.n = n;
  t.parent.assign(parent, parent + n);
  t.phys.assign(phys, phys + n);
  t.children.assign(n, {});
  for (int i = 0; i < n; ++i) {
    TTN_REQUIRE(phys[i] >= 0, "tree: phys_dim[%d] < 0", i);
    if (parent[i] < 0) {
      TTN_REQUIRE(t.root < 0, "tree: more than one root");
      TTN_REQUIRE(parent[i] == -1, "tree: parent[%d] must be -1 or a node", i);
      t.root = i;
    } else {
      TTN_REQUIRE(parent[i] < n && parent[i] != i, "tree: bad parent[%d] = %d", i, parent[i]);
      t.children[parent[i]].push_back(i);
    }
  }
  TTN_REQUIRE(t.root >= 0, "tree: no root");
  t.legs.assign(n, {});
  for (int i = 0; i < n; ++i) {
    if (parent[i] >= 0) t.legs[i].push_back(parent[i]);
    for (int c : t.children[i]) t.legs[i].push_back(c);
    TTN_REQUIRE(t.nlegs(i) <= TTN_MAX_LEGS - 1, "tree: node %d has too many legs", i);
  }
  std::vector<int> seen(n, 0);
  std::function<void(int)> rec = [&](int u) {
    seen[u] = 1;
    t.pre.push_back(u);
    for (int c : t.children[u]) rec(c);
    t.post.push_back(u);
  };
  rec(t.root);
  for (int i = 0; i < n; ++i) TTN_REQUIRE(seen[i], "tree: node %d not reachable from the root", i);
  return t;
}

// ------------------------------------------------------------------------------------------------
// TTNO builder (Sec. II.A.3): leaves-to-root sweep, per-edge bipartite graph of (subtree part,
// rest part) with proportional rows/columns merged and a minimum vertex cover (Koenig).
// ------------------------------------------------------------------------------------------------
namespace {

struct PTerm {
  double coef;
  std::vector<std::pair<int, int>> chans;  // (edge child node, channel)
  std::vector<std::pair<int, int>> ops;    // (node, op id)
};

using Row = std::map<int, double>;

// Groups of indices whose rows are proportional (same support, equal ratios within tol).
std::vector<std::vector<int>> proportional_groups(const std::vector<Row>& rows, double tol) {
  std::map<std::vector<int>, std::vector<int>> by_support;
  for (int i = 0; i < (int)rows.size(); ++i) {
    std::vector<int> sup;
    for (auto& kv : rows[i]) sup.push_back(kv.first);
    by_support[sup].push_back(i);
  }
  std::vector<std::vector<int>> groups;
  for (auto& kv : by_support) {
    std::vector<int> members = kv.second;
    std::vector<char> used(members.size(), 0);
    for (size_t a = 0; a < members.size(); ++a) {
      if (used[a]) continue;
      std::vector<int> g{members[a]};
      used[a] = 1;
      const Row& ra = rows[members[a]];
      const double na = ra.begin()->second;
      for (size_t b = a + 1; b < members.size(); ++b) {
        if (used[b]) continue;
        const Row& rb = rows[members[b]];
        const double nb = rb.begin()->second;
        bool prop = true;
        for (auto ia = ra.begin(), ib = rb.begin(); ia != ra.end(); ++ia, ++ib) {
          const double x = ia->second / na, y = ib->second / nb;
          if (std::fabs(x - y) > tol * std::max(std::fabs(x), std::fabs(y))) {
            prop = false;
            break;
          }
        }
        if (prop) {
          g.push_back(members[b]);
          used[b] = 1;
        }
      }
      groups.push_back(g);
    }
  }
  std::sort(groups.begin(), groups.end());
  return groups;
}

// Minimum vertex cover of a bipartite graph (adj: left -> rights) via a maximum matching
// (augmenting paths) and Koenig's construction.
void min_vertex_cover(int nL, int nR, const std::vector<std::vector<int>>& adj,
                      std::vector<char>& coverL, std::vector<char>& coverR) {
  std::vector<int> matchR(nR, -1), matchL(nL, -1);
  std::vector<int> vis(nR, -1);
  std::function<bool(int, int)> aug = [&](int u, int stamp) -> bool {
    for (int v : adj[u]) {
      if (vis[v] == stamp) continue;
      vis[v] = stamp;
      if (matchR[v] < 0 || aug(matchR[v], stamp)) {
        matchR[v] = u;
        matchL[u] = v;
        return true;
      }
    }
    return false;
  };
  for (int u = 0; u < nL; ++u) aug(u, u);
  std::vector<char> zL(nL, 0), zR(nR, 0);
  std::vector<int> stack;
  for (int u = 0; u < nL; ++u)
    if (matchL[u] < 0) {
      zL[u] = 1;
      stack.push_back(u);
    }
  while (!stack.empty()) {
    const int u = stack.back();
    stack.pop_back();
    for (int v : adj[u]) {
      if (zR[v] || matchL[u] == v) continue;
      zR[v] = 1;
      const int w = matchR[v];
      if (w >= 0 && !zL[w]) {
        zL[w] = 1;
        stack.push_back(w);
      }
    }
  }
  coverL.assign(nL, 0);
  coverR.assign(nR, 0);
  for (int u = 0; u < nL; ++u) coverL[u] = !zL[u];
  for (int v = 0; v < nR; ++v) coverR[v] = zR[v];
}

}  // namespace

static int identity_op(ttn_ttno* H, std::vector<int>& id_op, int node) {
  if (id_op[node] >= 0) return id_op[node];
  const int d = H->tree.d(node);
  id_op[node] = (int)H->op_node.size();
  H->op_node.push_back(node);
  for (int p = 0; p < d; ++p)
    for (int q = 0; q < d; ++q) H->op_data.push_back(p == q ? 1.0 : 0.0);
  H->op_off.push_back((long long)H->op_data.size());
  return id_op[node];
}

static void copy_op_table(ttn_ttno* H, int n_ops, const int* op_site, const long long* op_offset,
                          const double* op_data) {
  TTN_REQUIRE(n_ops >= 0 && (n_ops == 0 || (op_site && op_offset && op_data)), "op table");
  H->op_off.assign(1, 0);
  for (int o = 0; o < n_ops; ++o) {
    const int s = op_site[o];
    TTN_REQUIRE(s >= 0 && s < H->tree.n, "op %d: bad site %d", o, s);
    const int d = H->tree.d(s);
    TTN_REQUIRE(op_offset[o + 1] - op_offset[o] == (long long)d * d,
                "op %d: expected %d x %d values", o, d, d);
    H->op_node.push_back(s);
    H->op_data.insert(H->op_data.end(), op_data + op_offset[o], op_data + op_offset[o + 1]);
    H->op_off.push_back((long long)H->op_data.size());
  }
}

// Numerical rank of a dense rows x cols matrix (row-major, destroyed): Householder QR with
// column pivoting in float64; columns whose remaining norm falls to tol * (largest column norm)
// or below end the factorisation.
static int pivoted_qr_rank(std::vector<double>& A, int rows, int cols, double tol) {
  std::vector<double> cn(cols, 0.0);
  for (int j = 0; j < cols; ++j)
    for (int i = 0; i < rows; ++i) cn[j] += A[(size_t)i * cols + j] * A[(size_t)i * cols + j];
  double first = 0.0;
  int r = 0;
  const int kmax = std::min(rows, cols);
  for (int k = 0; k < kmax; ++k) {
    int p = k;
    for (int j = k + 1; j < cols; ++j)
      if (cn[j] > cn[p]) p = j;
    if (p != k) {
      std::swap(cn[p], cn[k]);
      for (int i = 0; i < rows; ++i) std::swap(A[(size_t)i * cols + p], A[(size_t)i * cols + k]);
    }
    double nrm = 0.0;   // recomputed from the trailing column (no downdating drift)
    for (int i = k; i < rows; ++i) nrm += A[(size_t)i * cols + k] * A[(size_t)i * cols + k];
    nrm = std::sqrt(nrm);
    if (k == 0) first = nrm;
    if (nrm <= tol * first || nrm == 0.0) break;
    ++r;
    const double a0 = A[(size_t)k * cols + k];
    const double alpha = a0 >= 0.0 ? -nrm : nrm;
    std::vector<double> v(rows - k);
    v[0] = a0 - alpha;
    for (int i = k + 1; i < rows; ++i) v[i - k] = A[(size_t)i * cols + k];
    double vv = 0.0;
    for (double x : v) vv += x * x;
    if (vv == 0.0) continue;
    for (int j = k; j < cols; ++j) {
      double dot = 0.0;
      for (int i = k; i < rows; ++i) dot += v[i - k] * A[(size_t)i * cols + j];
      const double f = 2.0 * dot / vv;
      for (int i = k; i < rows; ++i) A[(size_t)i * cols + j] -= f * v[i - k];
    }
    for (int j = k + 1; j < cols; ++j) {
      double s2 = 0.0;
      for (int i = k + 1; i < rows; ++i) s2 += A[(size_t)i * cols + j] * A[(size_t)i * cols + j];
      cn[j] = s2;
    }
  }
  return r;
}

// For every edge (child node c): the terms split into the operator string on the subtree of c
// and the string on the rest of the tree; the coefficient matrix C[subtree string][rest string]
// (sum of the coefficients of the terms with those two parts) has the smallest bond any exact
// TTNO of H can have on that edge as its rank, when distinct strings are linearly independent
// operators. The rank is taken by pivoted QR with a relative tolerance of 1e-12.
static std::vector<int> edge_rank_bounds(const TreeInfo& tree, int n_terms, const double* coeff,
                                         const int* term_offset, const int* term_op_ids,
                                         const int* op_site) {
  std::vector<int> out(tree.n, 1);
  for (int c = 0; c < tree.n; ++c) {
    if (c == tree.root) continue;
    std::vector<char> in_sub(tree.n, 0);
    std::vector<int> st{c};
    while (!st.empty()) {
      const int u = st.back();
      st.pop_back();
      in_sub[u] = 1;
      for (int ch : tree.children[u]) st.push_back(ch);
    }
    std::map<std::vector<int>, int> L, R;
    std::vector<std::tuple<int, int, double>> nz;
    for (int t = 0; t < n_terms; ++t) {
      if (coeff[t] == 0.0) continue;
      std::vector<int> l, r;
      for (int k = term_offset[t]; k < term_offset[t + 1]; ++k)
        (in_sub[op_site[term_op_ids[k]]] ? l : r).push_back(term_op_ids[k]);
      std::sort(l.begin(), l.end());
      std::sort(r.begin(), r.end());
      const int li = L.emplace(l, (int)L.size()).first->second;
      const int ri = R.emplace(r, (int)R.size()).first->second;
      nz.emplace_back(li, ri, coeff[t]);
    }
    const int rows = (int)L.size(), cols = (int)R.size();
    if (rows == 0 || cols == 0) {
      out[c] = 0;
      continue;
    }
    std::vector<double> A((size_t)rows * cols, 0.0);
    for (auto& e : nz) A[(size_t)std::get<0>(e) * cols + std::get<1>(e)] += std::get<2>(e);
    out[c] = pivoted_qr_rank(A, rows, cols, 1e-12);
  }
  return out;
}

static ttn_ttno* build_ttno_impl(ttn_ctx* ctx, const TreeInfo& tree, int n_ops,
                                 const int* op_site, const long long* op_offset,
                                 const double* op_data, int n_terms, const double* coeff,
                                 const int* term_offset, const int* term_op_ids, double tol) {
  auto H = std::make_unique<ttn_ttno>();
  H->ctx = ctx;
  H->tree = tree;
  copy_op_table(H.get(), n_ops, op_site, op_offset, op_data);
  for (int o = 0; o < n_ops; ++o)
    TTN_REQUIRE(tree.phys[op_site[o]] > 0, "op %d sits on an auxiliary node", o);
  TTN_REQUIRE(n_terms >= 0 && (n_terms == 0 || (coeff && term_offset && term_op_ids)), "terms");
  const int n = tree.n;
  std::vector<int> id_op(n, -1);
  std::vector<PTerm> terms;
  for (int t = 0; t < n_terms; ++t) {
    PTerm pt;
    pt.coef = coeff[t];
    for (int k = term_offset[t]; k < term_offset[t + 1]; ++k) {
      const int o = term_op_ids[k];
      TTN_REQUIRE(o >= 0 && o < n_ops, "term %d: bad op id %d", t, o);
      pt.ops.push_back({op_site[o], o});
    }
    std::sort(pt.ops.begin(), pt.ops.end());
    for (size_t k = 1; k < pt.ops.size(); ++k)
      TTN_REQUIRE(pt.ops[k].first != pt.ops[k - 1].first, "term %d: two ops on one node", t);
    if (pt.coef != 0.0) terms.push_back(pt);
  }
  H->wbond.assign(n, 1);
  H->entries.assign(n, {});
  for (int t : tree.post) {
    const std::vector<int>& ch = tree.children[t];
    const bool root = t == tree.root;
    // split every term into (left key, right key)
    std::map<std::vector<int>, int> Lidx, Ridx;
    std::vector<std::vector<int>> Lkeys, Rkeys;
    std::vector<Row> rows;
    for (const PTerm& pt : terms) {
      std::vector<int> lk(ch.size(), -1), rk;
      int opt = -1;
      std::vector<std::pair<int, int>> rch, rops;
      for (auto& c : pt.chans) {
        auto it = std::find(ch.begin(), ch.end(), c.first);
        if (it != ch.end()) lk[it - ch.begin()] = c.second;
        else rch.push_back(c);
      }
      for (auto& o : pt.ops) {
        if (o.first == t) opt = o.second;
        else rops.push_back(o);
      }
      for (size_t m = 0; m < ch.size(); ++m)
        TTN_REQUIRE(lk[m] >= 0, "internal: term without a channel on edge %d", ch[m]);
      lk.push_back(opt < 0 ? identity_op(H.get(), id_op, t) : opt);
      rk.push_back((int)rch.size());
      for (auto& c : rch) {
        rk.push_back(c.first);
        rk.push_back(c.second);
      }
      for (auto& o : rops) {
        rk.push_back(o.first);
        rk.push_back(o.second);
      }
      auto li = Lidx.emplace(lk, (int)Lkeys.size());
      if (li.second) {
        Lkeys.push_back(lk);
        rows.emplace_back();
      }
      auto ri = Ridx.emplace(rk, (int)Rkeys.size());
      if (ri.second) Rkeys.push_back(rk);
      rows[li.first->second][ri.first->second] += pt.coef;
    }
    for (Row& r : rows)
      for (auto it = r.begin(); it != r.end();)
        it = it->second == 0.0 ? r.erase(it) : std::next(it);
    auto emit = [&](int w0, const std::vector<int>& lk, double coef) {
      TtnoEntry e{};
      int m = 0;
      if (!root) e.w[m++] = w0;
      for (size_t k = 0; k + 1 < lk.size(); ++k) e.w[m++] = lk[k];
      e.op = lk.back();
      e.coef = coef;
      H->entries[t].push_back(e);
    };
    if (root) {
      for (size_t l = 0; l < Lkeys.size(); ++l) {
        double c = 0.0;
        for (auto& kv : rows[l]) c += kv.second;   // right key is empty at the root
        if (c != 0.0) emit(0, Lkeys[l], c);
      }
      break;
    }
    const int nL = (int)Lkeys.size(), nR = (int)Rkeys.size();
    std::vector<Row> cols(nR);
    for (int l = 0; l < nL; ++l)
      for (auto& kv : rows[l]) cols[kv.first][l] = kv.second;
    std::vector<int> active_l, active_r;
    std::vector<Row> arows, acols;
    for (int l = 0; l < nL; ++l)
      if (!rows[l].empty()) {
        active_l.push_back(l);
        arows.push_back(rows[l]);
      }
    for (int r = 0; r < nR; ++r)
      if (!cols[r].empty()) {
        active_r.push_back(r);
        acols.push_back(cols[r]);
      }
    auto GL = proportional_groups(arows, tol);
    auto GR = proportional_groups(acols, tol);
    for (auto& g : GL)
      for (int& x : g) x = active_l[x];
    for (auto& g : GR)
      for (int& x : g) x = active_r[x];
    std::vector<int> gl_of(nL, -1), gr_of(nR, -1);
    for (int g = 0; g < (int)GL.size(); ++g)
      for (int x : GL[g]) gl_of[x] = g;
    for (int g = 0; g < (int)GR.size(); ++g)
      for (int x : GR[g]) gr_of[x] = g;
    std::vector<std::vector<int>> adj(GL.size());
    for (int g = 0; g < (int)GL.size(); ++g) {
      std::set<int> s;
      for (int l : GL[g])
        for (auto& kv : rows[l]) s.insert(gr_of[kv.first]);
      adj[g].assign(s.begin(), s.end());
    }
    std::vector<char> cL, cR;
    min_vertex_cover((int)GL.size(), (int)GR.size(), adj, cL, cR);
    std::map<std::vector<std::pair<int, int>>, std::map<std::vector<std::pair<int, int>>, double>>
        merged;  // chans -> ops -> coef
    auto continue_term = [&](int r, int chan, double coef) {
      const std::vector<int>& rk = Rkeys[r];
      std::vector<std::pair<int, int>> chans, ops;
      int k = 1;
      for (int i = 0; i < rk[0]; ++i, k += 2) chans.push_back({rk[k], rk[k + 1]});
      for (; k < (int)rk.size(); k += 2) ops.push_back({rk[k], rk[k + 1]});
      chans.push_back({t, chan});
      std::sort(chans.begin(), chans.end());
      merged[chans][ops] += coef;
    };
    int nchan = 0;
    std::vector<char> l_covered(nL, 0);
    for (int g = 0; g < (int)GL.size(); ++g) {
      if (!cL[g]) continue;
      const int c = nchan++;
      const int l0 = GL[g][0];
      const int r0 = rows[l0].begin()->first;
      const double n0 = rows[l0].begin()->second;
      for (int l : GL[g]) {
        l_covered[l] = 1;
        emit(c, Lkeys[l], rows[l].at(r0) / n0);
      }
      for (auto& kv : rows[l0]) continue_term(kv.first, c, kv.second);
    }
    for (int g = 0; g < (int)GR.size(); ++g) {
      if (!cR[g]) continue;
      const int r0 = GR[g][0];
      std::vector<std::pair<int, double>> kappa;
      for (auto& kv : cols[r0])
        if (!l_covered[kv.first]) kappa.push_back(kv);
      if (kappa.empty()) continue;
      const int c = nchan++;
      const int lref = cols[r0].begin()->first;
      const double nref = cols[r0].begin()->second;
      for (auto& kv : kappa) emit(c, Lkeys[kv.first], kv.second);
      for (int r : GR[g]) continue_term(r, c, cols[r].at(lref) / nref);
    }
    H->wbond[t] = std::max(nchan, 1);
    terms.clear();
    for (auto& a : merged)
      for (auto& b : a.second)
        if (b.second != 0.0) terms.push_back({b.second, a.first, b.first});
  }
  return H.release();
}

ttn_ttno* identity_ttno(ttn_ctx* ctx, const TreeInfo& tree) {
  auto H = std::make_unique<ttn_ttno>();
  H->ctx = ctx;
  H->tree = tree;
  H->wbond.assign(tree.n, 1);
  H->entries.assign(tree.n, {});
  H->op_off.assign(1, 0);
  std::vector<int> id_op(tree.n, -1);
  for (int t = 0; t < tree.n; ++t) {
    TtnoEntry e{};
    e.op = identity_op(H.get(), id_op, t);
    e.coef = 1.0;
    H->entries[t].push_back(e);
  }
  return H.release();
}

// ------------------------------------------------------------------------------------------------
// blocks
// ------------------------------------------------------------------------------------------------
const float* ttn_block::node32(int t) const {
  if (!f32_valid) {
    if (!d32.p) d32 = DevBuf((size_t)total * sizeof(float), ctx->stream);
    launch_to_f32(ctx, d64.as<double>(), d32.as<float>(), total);
    f32_valid = true;
  }
  return d32.as<float>() + off[t];
}

static ttn_block* make_block(ttn_ctx* ctx, const TreeInfo& tree, int n_states, const int* bond) {
  TTN_REQUIRE(n_states >= 0 && bond, "block: bad arguments");
  auto b = std::make_unique<ttn_block>();
  b->ctx = ctx;
  b->tree = tree;
  b->n_states = n_states;
  b->bond.assign(bond, bond + tree.n);
  b->bond[tree.root] = 1;
  for (int i = 0; i < tree.n; ++i)
    TTN_REQUIRE(b->bond[i] >= 1, "block: bond_dims[%d] = %d must be >= 1", i, b->bond[i]);
  b->dims.assign(tree.n, {});
  b->size.assign(tree.n, 0);
  b->off.assign(tree.n, 0);
  long long off = 0;
  for (int t = 0; t < tree.n; ++t) {
    long long sz = tree.d(t);
    for (int m = 0; m < tree.nlegs(t); ++m) {
      b->dims[t].push_back(b->bdim(t, m));
      sz *= b->bdim(t, m);
    }
    b->dims[t].push_back(tree.d(t));
    b->size[t] = sz;
    b->off[t] = off;
    off += sz * n_states;
  }
  b->total = off;
  b->d64 = DevBuf((size_t)std::max<long long>(off, 1) * sizeof(double), ctx->stream);
  CUDA_CHECK(cudaMemsetAsync(b->d64.p, 0, (size_t)std::max<long long>(off, 1) * sizeof(double),
                             ctx->stream));
  return b.release();
}

void iter_clock_start(ttn_ctx* ctx) {
  ctx->iter_marks = -1;
  iter_clock_mark(ctx);
}

void iter_clock_mark(ttn_ctx* ctx) {
  const size_t i = (size_t)(ctx->iter_marks + 1);
  while (ctx->iter_ev.size() <= i) {
    cudaEvent_t e;
    CUDA_CHECK(cudaEventCreate(&e));
    ctx->iter_ev.push_back(e);
  }
  CUDA_CHECK(cudaEventRecord(ctx->iter_ev[i], ctx->stream));
  ctx->iter_marks = (int)i;
}

// ------------------------------------------------------------------------------------------------
// C ABI helpers
// ------------------------------------------------------------------------------------------------
// Reports (once) a bounded device-side wait that gave up in work issued earlier on the context.
static void raise_wait_timeout(ttn_ctx* ctx) {
  if (!ctx || !ctx->h_wait) return;
  volatile unsigned* f = ctx->h_wait;
  const unsigned v = *f;
  if (v == 0u) return;
  *f = 0u;
  if (v == TTN_WAIT_FLAG_SELFTEST)
    TTN_FAIL(TTN_ETIMEOUT, "bounded-wait self-test: the barrier wait gave up as intended (no "
                           "copy was in flight; the context stays usable)");
  if (v == TTN_WAIT_FLAG_MMA)
    TTN_FAIL(TTN_ETIMEOUT, "a wait for tensor-core MMA completion on the device gave up after "
                           "2 s; results of the work issued since the previous call are not valid "
                           "and the context must be destroyed");
  TTN_FAIL(TTN_ETIMEOUT, "a bulk-copy barrier wait on the device gave up after 2 s; copies may "
                         "still have been landing when the waiting block left, so results of the "
                         "work issued since the previous call are not valid and the context must "
                         "be destroyed");
}

template <class F>
static ttn_status guarded(ttn_ctx* ctx, F&& f) {
  try {
    f();
    raise_wait_timeout(ctx);
    if (ctx) ctx->last_error.clear();
    return TTN_OK;
  } catch (const TtnError& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return TTN_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what();
    return TTN_EINVAL;
  }
}

struct DevInts {
  DevBuf buf;
  int maxv = 0;
  DevInts(const std::vector<int>& v, cudaStream_t s)
      : buf(std::max<size_t>(v.size(), 1) * sizeof(int), s) {
    for (int x : v) maxv = std::max(maxv, x);
    if (!v.empty())
      CUDA_CHECK(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 s));
    CUDA_CHECK(cudaStreamSynchronize(s));
  }
  const int* get() const { return buf.as<int>(); }
};

static ttn_ttno* cached_identity(ttn_ctx* ctx, const TreeInfo& tree);

// ------------------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------------------
// Identity TTNOs per context, released by ttn_destroy. The map itself is never destroyed: a
// static destructor running after the CUDA runtime has been torn down at process exit must not
// touch device memory.
struct IdCache {
  std::vector<std::pair<TreeInfo, ttn_ttno*>> items;
  void release() {
    for (auto& it : items) delete it.second;
    items.clear();
  }
};
static std::map<const ttn_ctx*, IdCache>& id_caches() {
  static auto* m = new std::map<const ttn_ctx*, IdCache>();
  return *m;
}

static ttn_ttno* cached_identity(ttn_ctx* ctx, const TreeInfo& tree) {
  IdCache& c = id_caches()[ctx];
  for (auto& it : c.items)
    if (it.first.same_shape(tree)) return it.second;
  ttn_ttno* H = identity_ttno(ctx, tree);
  c.items.push_back({tree, H});
  return H;
}

extern "C" {

ttn_status ttn_create(ttn_ctx** out, int device, void* cuda_stream) {
  if (!out) return TTN_EINVAL;
  *out = nullptr;
  auto ctx = std::make_unique<ttn_ctx>();
  ttn_status st = guarded(ctx.get(), [&] {
    if (device == -1) {   // host-only context: trees and TTNO construction/export only
      ctx->device = -1;
      return;
    }
    int n = 0;
    CUDA_CHECK(cudaGetDeviceCount(&n));
    TTN_REQUIRE(device >= 0 && device < n, "device %d not present (%d devices)", device, n);
    CUDA_CHECK(cudaSetDevice(device));
    ctx->device = device;
    CUDA_CHECK(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    void* hw = nullptr;
    CUDA_CHECK(cudaHostAlloc(&hw, sizeof(unsigned), cudaHostAllocMapped));
    ctx->h_wait = static_cast<unsigned*>(hw);
    *ctx->h_wait = 0u;
    void* dw = nullptr;
    CUDA_CHECK(cudaHostGetDevicePointer(&dw, hw, 0));
    ctx->d_wait = static_cast<unsigned*>(dw);
    if (const char* lp = getenv("TTN_LAUNCH_LOG")) ctx->launch_log = std::fopen(lp, "a");
    rr_noalloc_prepare(device);
    cudaMemPool_t pool;
    CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  });
  if (st == TTN_OK) *out = ctx.release();
  return st;
}

void ttn_destroy(ttn_ctx* ctx) {
  if (!ctx) return;
  if (ctx->device < 0) {
    delete ctx;
    return;
  }
  cudaStreamSynchronize(ctx->stream);
  auto it = id_caches().find(ctx);
  if (it != id_caches().end()) {
    it->second.release();
    id_caches().erase(it);
  }
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->prof) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  for (auto e : ctx->iter_ev) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->h_wait) cudaFreeHost(ctx->h_wait);
  if (ctx->launch_log) std::fclose(ctx->launch_log);
  delete ctx;
}

const char* ttn_last_error(const ttn_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

ttn_status ttn_synchronize(ttn_ctx* ctx) {
  if (!ctx) return TTN_EINVAL;
  return guarded(ctx, [&] { CUDA_CHECK(cudaStreamSynchronize(ctx->stream)); });
}

ttn_status ttn_selftest_bounded_wait(ttn_ctx* ctx, double budget_ms) {
  if (!ctx) return TTN_EINVAL;
  return guarded(ctx, [&] {
    TTN_REQUIRE(ctx->device >= 0, "a host-only context has no device");
    TTN_REQUIRE(budget_ms >= 0.001 && budget_ms <= 1000.0,
                "budget_ms = %g outside [0.001, 1000]", budget_ms);
    launch_wait_selftest(ctx, (unsigned long long)(budget_ms * 1e6));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  });
}

void ttn_fault_inject_alloc(long long after) { g_alloc_countdown.store(after < 0 ? -1 : after); }

int ttn_iteration_times(ttn_ctx* ctx, double* ms, int max_n) {
  if (!ctx || ctx->device < 0 || ctx->iter_marks < 1) return 0;
  if (cudaEventSynchronize(ctx->iter_ev[ctx->iter_marks]) != cudaSuccess) return -1;
  const int n = ctx->iter_marks;
  for (int i = 0; i < n && i < max_n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->iter_ev[0], ctx->iter_ev[i + 1]) != cudaSuccess) return -1;
    ms[i] = t;
  }
  return n;
}

long long ttn_launch_count(const ttn_ctx* ctx) { return ctx ? ctx->launches : 0; }

double ttn_flop_count(const ttn_ctx* ctx) { return ctx ? ctx->flops_total : 0.0; }

ttn_status ttn_profile_enable(ttn_ctx* ctx, int on) {
  if (!ctx) return TTN_EINVAL;
  return guarded(ctx, [&] {
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    for (auto& r : ctx->prof) {
      ctx->event_pool.push_back(r.start);
      ctx->event_pool.push_back(r.stop);
    }
    ctx->prof.clear();
    ctx->profiling = on != 0;
  });
}

ttn_status ttn_profile_get(ttn_ctx* ctx, int max_kernels, char* names, long long* launches,
                           double* ms, double* flops, double* bytes, int* n_kernels) {
  if (!ctx || !n_kernels) return TTN_EINVAL;
  return guarded(ctx, [&] {
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    const int nk = (int)ctx->prof_names.size();
    std::vector<long long> cnt(nk, 0);
    std::vector<double> t(nk, 0.0), f(nk, 0.0), b(nk, 0.0);
    for (auto& r : ctx->prof) {
      float e = 0.f;
      CUDA_CHECK(cudaEventElapsedTime(&e, r.start, r.stop));
      cnt[r.name]++;
      t[r.name] += e;
      f[r.name] += r.flops;
      b[r.name] += r.bytes;
    }
    *n_kernels = nk;
    for (int i = 0; i < nk && i < max_kernels; ++i) {
      if (names) {
        std::strncpy(names + 64 * i, ctx->prof_names[i].c_str(), 63);
        names[64 * i + 63] = 0;
      }
      if (launches) launches[i] = cnt[i];
      if (ms) ms[i] = t[i];
      if (flops) flops[i] = f[i];
      if (bytes) bytes[i] = b[i];
    }
  });
}

// ------------------------------------------------------------------------------------------------
// tree / TTNO
// ------------------------------------------------------------------------------------------------
ttn_status ttn_tree_create(ttn_ctx* ctx, int n_nodes, const int* parent, const int* phys_dim,
                           ttn_tree** out) {
  if (!ctx || !out) return TTN_EINVAL;
  return guarded(ctx, [&] {
    TreeInfo t = make_tree(n_nodes, parent, phys_dim);
    auto* tr = new ttn_tree;
    tr->info = std::move(t);
    tr->ctx = ctx;
    *out = tr;
  });
}

void ttn_tree_destroy(ttn_tree* tree) { delete tree; }

ttn_status ttn_build_ttno(ttn_ctx* ctx, const ttn_tree* tree, int n_ops, const int* op_site,
                          const long long* op_offset, const double* op_data, int n_terms,
                          const double* coeff, const int* term_offset, const int* term_op_ids,
                          double tol, ttn_ttno** out, int* bond_dims_out) {
  if (!ctx || !tree || !out) return TTN_EINVAL;
  return guarded(ctx, [&] {
    TTN_REQUIRE(tol >= 0.0, "tol must be >= 0");
    ttn_ttno* H = build_ttno_impl(ctx, tree->info, n_ops, op_site, op_offset, op_data, n_terms,
                                  coeff, term_offset, term_op_ids, tol);
    H->rank_bound = edge_rank_bounds(tree->info, n_terms, coeff, term_offset, term_op_ids,
                                     op_site);
    if (bond_dims_out)
      for (int i = 0; i < tree->info.n; ++i) bond_dims_out[i] = H->wbond[i];
    *out = H;
  });
}

ttn_status ttn_ttno_create(ttn_ctx* ctx, const ttn_tree* tree, const int* wbond, int n_ops,
                           const int* op_site, const long long* op_offset,
                           const double* op_data, int n_entries, const int* entry_node,
                           const int* entry_w, const int* entry_op, const double* entry_coef,
                           ttn_ttno** out) {
  if (!ctx || !tree || !out || !wbond) return TTN_EINVAL;
  return guarded(ctx, [&] {
    auto H = std::make_unique<ttn_ttno>();
    H->ctx = ctx;
    H->tree = tree->info;
    const TreeInfo& tr = H->tree;
    H->wbond.assign(wbond, wbond + tr.n);
    H->wbond[tr.root] = 1;
    for (int i = 0; i < tr.n; ++i) TTN_REQUIRE(H->wbond[i] >= 1, "wbond[%d] < 1", i);
    copy_op_table(H.get(), n_ops, op_site, op_offset, op_data);
    H->entries.assign(tr.n, {});
    TTN_REQUIRE(n_entries >= 0 && (n_entries == 0 || (entry_node && entry_w && entry_op &&
                                                       entry_coef)),
                "entries");
    for (int e = 0; e < n_entries; ++e) {
      const int t = entry_node[e];
      TTN_REQUIRE(t >= 0 && t < tr.n, "entry %d: bad node", e);
      TtnoEntry en{};
      for (int m = 0; m < tr.nlegs(t); ++m) {
        en.w[m] = entry_w[(long long)e * TTN_MAX_LEGS + m];
        TTN_REQUIRE(en.w[m] >= 0 && en.w[m] < H->wdim(t, m), "entry %d: w[%d] out of range", e,
                    m);
      }
      en.op = entry_op[e];
      TTN_REQUIRE(en.op >= 0 && en.op < n_ops && H->op_node[en.op] == t,
                  "entry %d: op %d is not an op of node %d", e, en.op, t);
      en.coef = entry_coef[e];
      H->entries[t].push_back(en);
    }
    *out = H.release();
  });
}

ttn_status ttn_ttno_rank_bounds(const ttn_ttno* H, int* rank_out) {
  if (!H || !rank_out) return TTN_EINVAL;
  for (int i = 0; i < H->tree.n; ++i)
    rank_out[i] = i < (int)H->rank_bound.size() ? H->rank_bound[i] : -1;
  return TTN_OK;
}

ttn_status ttn_ttno_info(const ttn_ttno* H, int* wbond_out, int* n_entries_out,
                         long long* n_op_doubles_out) {
  if (!H) return TTN_EINVAL;
  long long ne = 0, nd = 0;
  for (int t = 0; t < H->tree.n; ++t) {
    ne += (long long)H->entries[t].size();
    const long long d = H->tree.d(t);
    nd += (long long)H->entries[t].size() * d * d;
  }
  if (wbond_out)
    for (int i = 0; i < H->tree.n; ++i) wbond_out[i] = H->wbond[i];
  if (n_entries_out) *n_entries_out = (int)ne;
  if (n_op_doubles_out) *n_op_doubles_out = nd;
  return TTN_OK;
}

ttn_status ttn_ttno_get_entries(const ttn_ttno* H, int* entry_node, int* entry_w,
                                double* entry_coef, long long* op_offset, double* op_data) {
  if (!H) return TTN_EINVAL;
  long long e = 0, od = 0;
  for (int t = 0; t < H->tree.n; ++t) {
    const int d = H->tree.d(t);
    for (const TtnoEntry& en : H->entries[t]) {
      if (entry_node) entry_node[e] = t;
      if (entry_w)
        for (int m = 0; m < TTN_MAX_LEGS; ++m)
          entry_w[e * TTN_MAX_LEGS + m] = m < H->tree.nlegs(t) ? en.w[m] : 0;
      if (entry_coef) entry_coef[e] = en.coef;
      if (op_offset) op_offset[e] = od;
      if (op_data)
        std::memcpy(op_data + od, H->op_data.data() + H->op_off[en.op],
                    sizeof(double) * d * d);
      od += (long long)d * d;
      ++e;
    }
  }
  if (op_offset) op_offset[e] = od;
  return TTN_OK;
}

void ttn_ttno_destroy(ttn_ttno* H) {
  if (!H) return;
  if (H->ctx->device >= 0) cudaStreamSynchronize(H->ctx->stream);
  delete H;
}

// ------------------------------------------------------------------------------------------------
// blocks
// ------------------------------------------------------------------------------------------------
ttn_status ttn_block_create(ttn_ctx* ctx, const ttn_tree* tree, int n_states,
                            const int* bond_dims, ttn_block** out) {
  if (!ctx || !tree || !out) return TTN_EINVAL;
  return guarded(ctx, [&] {
    TTN_REQUIRE(ctx->device >= 0, "a host-only context (device -1) cannot hold device blocks");
    *out = make_block(ctx, tree->info, n_states, bond_dims); });
}

void ttn_block_destroy(ttn_block* b) {
  if (!b) return;
  cudaStreamSynchronize(b->ctx->stream);
  delete b;
}

ttn_status ttn_block_set(ttn_block* b, int state, int node, const double* host, long long n) {
  if (!b || !host) return TTN_EINVAL;
  return guarded(b->ctx, [&] {
    TTN_REQUIRE(node >= 0 && node < b->tree.n, "bad node %d", node);
    TTN_REQUIRE(state >= -1 && state < b->n_states, "bad state %d", state);
    const long long want = state < 0 ? b->size[node] * b->n_states : b->size[node];
    TTN_REQUIRE(n == want, "node %d: expected %lld values, got %lld", node, want, n);
    double* dst = b->node64(node) + (state < 0 ? 0 : (long long)state * b->size[node]);
    CUDA_CHECK(cudaMemcpyAsync(dst, host, n * sizeof(double), cudaMemcpyHostToDevice,
                               b->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(b->ctx->stream));
    b->touch();
  });
}

ttn_status ttn_block_get(const ttn_block* b, int state, int node, double* host, long long n) {
  if (!b || !host) return TTN_EINVAL;
  return guarded(b->ctx, [&] {
    TTN_REQUIRE(node >= 0 && node < b->tree.n, "bad node %d", node);
    TTN_REQUIRE(state >= -1 && state < b->n_states, "bad state %d", state);
    const long long want = state < 0 ? b->size[node] * b->n_states : b->size[node];
    TTN_REQUIRE(n == want, "node %d: expected %lld values, got %lld", node, want, n);
    const double* src = b->node64(node) + (state < 0 ? 0 : (long long)state * b->size[node]);
    CUDA_CHECK(cudaMemcpyAsync(host, src, n * sizeof(double), cudaMemcpyDeviceToHost,
                               b->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(b->ctx->stream));
  });
}

ttn_status ttn_block_node_info(const ttn_block* b, int node, long long* size,
                               double** device_ptr) {
  if (!b || node < 0 || node >= b->tree.n) return TTN_EINVAL;
  if (size) *size = b->size[node];
  if (device_ptr) *device_ptr = b->node64(node);
  return TTN_OK;
}

ttn_status ttn_block_copy_states(ttn_block* dst, const ttn_block* src, int n,
                                 const int* src_states) {
  if (!dst || !src || (n > 0 && !src_states)) return TTN_EINVAL;
  return guarded(dst->ctx, [&] {
    TTN_REQUIRE(dst->tree.same_shape(src->tree) && dst->bond == src->bond,
                "copy_states: blocks differ in tree or bonds");
    TTN_REQUIRE(n <= dst->n_states, "copy_states: too many states");
    for (int j = 0; j < n; ++j)
      TTN_REQUIRE(src_states[j] >= 0 && src_states[j] < src->n_states, "bad source state");
    if (n == 0) return;
    TTN_REQUIRE(dst != src, "copy_states: source and destination are the same block");
    DevInts idx(std::vector<int>(src_states, src_states + n), dst->ctx->stream);
    for (int t = 0; t < dst->tree.n; ++t)     // one gather launch per node
      launch_gather_rows(dst->ctx, dst->node64(t), src->node64(t), idx.get(), n, dst->size[t]);
    dst->touch();
  });
}

// ------------------------------------------------------------------------------------------------
// environments
// ------------------------------------------------------------------------------------------------
ttn_status ttn_envs_create(ttn_ctx* ctx, const ttn_tree* tree, ttn_envs** out) {
  if (!ctx || !tree || !out) return TTN_EINVAL;
  return guarded(ctx, [&] {
    TTN_REQUIRE(ctx->device >= 0, "a host-only context (device -1) cannot hold environments");
    auto* e = new ttn_envs;
    e->ctx = ctx;
    e->tree = tree->info;
    *out = e;
  });
}

void ttn_envs_destroy(ttn_envs* e) {
  if (!e) return;
  cudaStreamSynchronize(e->ctx->stream);
  delete e;
}

static void check_pair_blocks(const ttn_ttno* H, const ttn_block* bra, const ttn_block* ket) {
  TTN_REQUIRE(bra && ket, "NULL block");
  TTN_REQUIRE(bra->tree.same_shape(ket->tree), "bra and ket blocks live on different trees");
  if (H) TTN_REQUIRE(H->tree.same_shape(bra->tree), "TTNO and blocks live on different trees");
}

ttn_status ttn_env_update(ttn_ctx* ctx, const ttn_ttno* Hc, const ttn_block* bra,
                          const ttn_block* ket, int n_pairs, const int* pair_bra,
                          const int* pair_ket, int direction, ttn_envs* envs,
                          ttn_precision prec) {
  if (!ctx || !envs) return TTN_EINVAL;
  return guarded(ctx, [&] {
    PrecisionScope prec_scope(ctx, prec);
    check_pair_blocks(Hc, bra, ket);
    TTN_REQUIRE(envs->tree.same_shape(bra->tree), "envs created for another tree");
    TTN_REQUIRE(direction >= 0 && direction <= 2, "direction must be 0, 1 or 2");
    TTN_REQUIRE(valid_precision(prec), "unknown precision %d", (int)prec);
    TTN_REQUIRE(n_pairs >= 0 && (n_pairs == 0 || (pair_bra && pair_ket)), "pairs");
    for (int i = 0; i < n_pairs; ++i)
      TTN_REQUIRE(pair_bra[i] >= 0 && pair_bra[i] < bra->n_states && pair_ket[i] >= 0 &&
                      pair_ket[i] < ket->n_states,
                  "pair %d out of range", i);
    ttn_ttno* H = Hc ? const_cast<ttn_ttno*>(Hc) : cached_identity(ctx, bra->tree);
    envs->n_pairs = n_pairs;
    envs->prec = prec;
    envs->H = H;
    envs->pair_bra.assign(pair_bra, pair_bra + n_pairs);
    envs->pair_ket.assign(pair_ket, pair_ket + n_pairs);
    const TreeInfo& tr = bra->tree;
    envs->Dw.assign(tr.n, 0);
    envs->Da.assign(tr.n, 0);
    envs->Db.assign(tr.n, 0);
    for (int c = 0; c < tr.n; ++c) {
      envs->Dw[c] = H->wbond[c];
      envs->Da[c] = bra->bond[c];
      envs->Db[c] = ket->bond[c];
    }
    envs->up.clear();
    envs->down.clear();
    if (n_pairs == 0) {
      envs->up.resize(tr.n);
      envs->down.resize(tr.n);
      envs->has_up = true;
      envs->has_down = direction != 0;
      return;
    }
    DevInts pb(envs->pair_bra, ctx->stream), pk(envs->pair_ket, ctx->stream);
    PairSet ps{n_pairs, pb.get(), pk.get(), pb.maxv, pk.maxv};
    if (prec == TTN_FP64)
      envs_compute<double>(ctx, H, bra, ket, ps, direction, envs->up, envs->down);
    else
      envs_compute<float>(ctx, H, bra, ket, ps, direction, envs->up, envs->down);
    envs->has_up = true;
    envs->has_down = direction != 0;
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  });
}

ttn_status ttn_envs_get(const ttn_envs* e, int node, int direction, int pair, double* host,
                        long long n) {
  if (!e || !host) return TTN_EINVAL;
  return guarded(e->ctx, [&] {
    TTN_REQUIRE(node >= 0 && node < e->tree.n && node != e->tree.root, "bad edge node %d", node);
    TTN_REQUIRE(pair >= 0 && pair < e->n_pairs, "bad pair %d", pair);
    TTN_REQUIRE((direction == 0 && e->has_up) || (direction == 1 && e->has_down),
                "direction %d not computed", direction);
    const long long sz = e->esize(node);
    TTN_REQUIRE(n == sz, "expected %lld values", sz);
    const DevBuf& b = direction == 0 ? e->up[node] : e->down[node];
    if (e->prec == TTN_FP64) {
      CUDA_CHECK(cudaMemcpyAsync(host, b.as<double>() + (long long)pair * sz, sz * sizeof(double),
                                 cudaMemcpyDeviceToHost, e->ctx->stream));
    } else {
      std::vector<float> tmp(sz);
      CUDA_CHECK(cudaMemcpyAsync(tmp.data(), b.as<float>() + (long long)pair * sz,
                                 sz * sizeof(float), cudaMemcpyDeviceToHost, e->ctx->stream));
      CUDA_CHECK(cudaStreamSynchronize(e->ctx->stream));
      for (long long i = 0; i < sz; ++i) host[i] = tmp[i];
    }
    CUDA_CHECK(cudaStreamSynchronize(e->ctx->stream));
  });
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// H_eff, Gram, apply (internal templated drivers used by the C ABI and the solvers)
// ------------------------------------------------------------------------------------------------
template <class T>
void heff_apply_impl(ttn_ctx* ctx, ttn_ttno* H, const ttn_envs* envs, int node, const ttn_block* x,
                     T* y_out, const int* d_id) {
  PairSet ps{x->n_states, d_id, d_id, x->n_states - 1, x->n_states - 1};
  const TreeInfo& tr = x->tree;
  const int nl = tr.nlegs(node);
  std::vector<const T*> env(nl, nullptr);
  std::vector<int> da(nl);
  for (int m = 0; m < nl; ++m) {
    const int nb = tr.legs[node][m];
    const int edge = tr.parent[node] == nb ? node : nb;
    env[m] = (tr.parent[node] == nb ? envs->down[edge] : envs->up[edge]).template as<T>();
    da[m] = envs->Da[edge];
  }
  long long ysize = x->tree.d(node);
  for (int m = 0; m < nl; ++m) ysize *= da[m];
  node_op<T>(ctx, H, node, -1, nullptr, x, ps, env, da, y_out, (long long)x->n_states * ysize,
             OUT_LOCAL);
}

template void heff_apply_impl<double>(ttn_ctx*, ttn_ttno*, const ttn_envs*, int,
                                      const ttn_block*, double*, const int*);
template void heff_apply_impl<float>(ttn_ctx*, ttn_ttno*, const ttn_envs*, int, const ttn_block*,
                                     float*, const int*);

// Bytes of device workspace one pair needs for the bottom-up sweep plus the root closure.
template <class T>
static long long gram_bytes_per_pair(ttn_ttno* H, const ttn_block* bra, const ttn_block* ket) {
  const TreeInfo& tr = bra->tree;
  long long envb = 0, inter = 0;
  for (int t = 0; t < tr.n; ++t) {
    if (t != tr.root) envb += (long long)H->wbond[t] * bra->bond[t] * ket->bond[t];
    const int open = t == tr.root ? -1 : 0;
    NodePlan& p = get_plan(H, t, open);
    long long sz = ket->size[t], tot = 0;
    for (size_t l = 0; l < p.C.size(); ++l) {
      const int c = p.C[l];
      sz = sz / ket->bdim(t, c) * bra->bdim(t, c);
      tot += sz * (long long)p.level[l].size();
    }
    tot += sz * p.n_slots;
    inter = std::max(inter, tot);
  }
  return (envb + inter) * (long long)sizeof(T) + 64;
}

// <bra_pb[i]| H |ket_pk[i]> for every listed pair, written to d_out[i] (device, float64).
template <class T>
void gram_pairs(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                const std::vector<int>& pb, const std::vector<int>& pk, double* d_out) {
  const int n_pairs = (int)pb.size();
  if (n_pairs == 0) return;
  const long long per = gram_bytes_per_pair<T>(H, bra, ket);
  const char* env_gb = getenv("TTN_WORKSPACE_GB");
  const double budget = (env_gb ? atof(env_gb) : 24.0) * 1e9;
  int chunk = (int)std::max<long long>(1, std::min<long long>(n_pairs, (long long)(budget / per)));
  const TreeInfo& tr = bra->tree;
  for (int c0 = 0; c0 < n_pairs; c0 += chunk) {
    const int P = std::min(chunk, n_pairs - c0);
    std::vector<int> cb(pb.begin() + c0, pb.begin() + c0 + P);
    std::vector<int> ck(pk.begin() + c0, pk.begin() + c0 + P);
    DevInts dpb(cb, ctx->stream), dpk(ck, ctx->stream);
    PairSet ps{P, dpb.get(), dpk.get(), dpb.maxv, dpk.maxv};
    std::vector<DevBuf> up, down;
    envs_compute<T>(ctx, H, bra, ket, ps, 0, up, down);
    const int nl = tr.nlegs(tr.root);
    std::vector<const T*> env(nl, nullptr);
    for (int m = 0; m < nl; ++m) env[m] = up[tr.legs[tr.root][m]].template as<T>();
    node_op<T>(ctx, H, tr.root, -1, bra, ket, ps, env, {}, d_out + c0, (long long)P, OUT_SCALAR);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  }
}

template void gram_pairs<double>(ttn_ctx*, ttn_ttno*, const ttn_block*, const ttn_block*,
                                 const std::vector<int>&, const std::vector<int>&, double*);
template void gram_pairs<float>(ttn_ctx*, ttn_ttno*, const ttn_block*, const ttn_block*,
                                const std::vector<int>&, const std::vector<int>&, double*);

// Writes the Gram of H into d_mat (device, leading dimension ld); returns the number of
// non-finite entries of the result.
unsigned gram_device(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                     double* d_mat, int ld, int prec) {
  const bool sym = bra == ket;
  std::vector<int> pb, pk;
  for (int k = 0; k < bra->n_states; ++k)
    for (int l = sym ? k : 0; l < ket->n_states; ++l) {
      pb.push_back(k);
      pk.push_back(l);
    }
  DevBuf g(std::max<size_t>(pb.size(), 1) * sizeof(double), ctx->stream);
  if (prec == TTN_FP64) gram_pairs<double>(ctx, H, bra, ket, pb, pk, g.as<double>());
  else gram_pairs<float>(ctx, H, bra, ket, pb, pk, g.as<double>());
  DevInts dpb(pb, ctx->stream), dpk(pk, ctx->stream);
  launch_scatter_gram(ctx, g.as<double>(), (int)pb.size(), dpb.get(), dpk.get(), sym ? 1 : 0,
                      d_mat, ld);
  DevBuf cnt(sizeof(unsigned), ctx->stream);
  launch_count_nonfinite(ctx, d_mat, bra->n_states, ket->n_states, ld, cnt.as<unsigned>());
  unsigned bad = 0;
  CUDA_CHECK(cudaMemcpyAsync(&bad, cnt.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  return bad;
}

ttn_ttno* identity_for(ttn_ctx* ctx, const TreeInfo& tree) { return cached_identity(ctx, tree); }

extern "C" {

ttn_status ttn_heff_apply(ttn_ctx* ctx, const ttn_ttno* Hc, const ttn_envs* envs, int node,
                          const ttn_block* x, ttn_block* y, const double* shift,
                          ttn_precision prec) {
  if (!ctx || !Hc || !envs || !x || !y) return TTN_EINVAL;
  return guarded(ctx, [&] {
    PrecisionScope prec_scope(ctx, prec);
    ttn_ttno* H = const_cast<ttn_ttno*>(Hc);
    check_pair_blocks(H, x, y);
    TTN_REQUIRE(node >= 0 && node < x->tree.n, "bad node");
    TTN_REQUIRE(envs->has_up && envs->has_down, "envs need both directions");
    TTN_REQUIRE(envs->H == H, "envs were computed with another operator");
    TTN_REQUIRE(envs->n_pairs == x->n_states && y->n_states == x->n_states,
                "envs pairs must match the states of x and y");
    TTN_REQUIRE(envs->prec == (int)prec, "envs were computed in another precision");
    for (int m = 0; m < x->tree.nlegs(node); ++m) {
      const int nb = x->tree.legs[node][m];
      const int edge = x->tree.parent[node] == nb ? node : nb;
      TTN_REQUIRE(envs->Db[edge] == x->bond[edge] && envs->Da[edge] == y->bond[edge],
                  "envs bonds do not match x/y on edge %d", edge);
    }
    std::vector<int> id(x->n_states);
    std::iota(id.begin(), id.end(), 0);
    DevInts did(id, ctx->stream);
    DevBuf dshift;
    if (shift) {
      dshift = DevBuf(std::max(x->n_states, 1) * sizeof(double), ctx->stream);
      CUDA_CHECK(cudaMemcpyAsync(dshift.p, shift, x->n_states * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream));
    }
    const long long sz = y->size[node];
    if (prec == TTN_FP64) {
      heff_apply_impl<double>(ctx, H, envs, node, x, y->node64(node), did.get());
      if (shift)
        launch_shift_axpy<double>(ctx, y->node64(node), x->node64(node), dshift.as<double>(),
                                  x->n_states, sz);
    } else {
      DevBuf tmp((size_t)x->n_states * sz * sizeof(float), ctx->stream);
      heff_apply_impl<float>(ctx, H, envs, node, x, tmp.as<float>(), did.get());
      if (shift)
        launch_shift_axpy<float>(ctx, tmp.as<float>(), x->node32(node), dshift.as<double>(),
                                 x->n_states, sz);
      launch_to_f64(ctx, tmp.as<float>(), y->node64(node), (long long)x->n_states * sz);
    }
    y->touch();
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  });
}

ttn_status ttn_gram(ttn_ctx* ctx, const ttn_ttno* Hc, const ttn_block* bra, const ttn_block* ket,
                    double* S, double* Hm, int ld, int out_on_device, ttn_precision prec) {
  if (!ctx || !bra || !ket) return TTN_EINVAL;
  return guarded(ctx, [&] {
    PrecisionScope prec_scope(ctx, prec);
    check_pair_blocks(Hc, bra, ket);
    TTN_REQUIRE(bra->bond == ket->bond || bra != ket, "internal");
    TTN_REQUIRE(ld >= ket->n_states, "ld < number of ket states");
    TTN_REQUIRE(valid_precision(prec), "unknown precision %d", (int)prec);
    const size_t mat = (size_t)bra->n_states * ld;
    unsigned bad = 0;
    auto one = [&](ttn_ttno* H, double* out) {
      if (!out) return;
      double* dst = out;
      DevBuf tmp;
      if (!out_on_device) {
        tmp = DevBuf(std::max<size_t>(mat, 1) * sizeof(double), ctx->stream);
        dst = tmp.as<double>();
      }
      CUDA_CHECK(cudaMemsetAsync(dst, 0, mat * sizeof(double), ctx->stream));
      bad += gram_device(ctx, H, bra, ket, dst, ld, prec);
      if (!out_on_device) {
        CUDA_CHECK(cudaMemcpyAsync(out, dst, mat * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
      }
    };
    if (Hm) TTN_REQUIRE(Hc, "Hm requested without an operator");
    one(cached_identity(ctx, bra->tree), S);
    if (Hm) one(const_cast<ttn_ttno*>(Hc), Hm);
    if (bad)
      TTN_FAIL(TTN_ENONFINITE, "%u Gram entries are NaN or infinite (results written)", bad);
  });
}

}  // extern "C"
