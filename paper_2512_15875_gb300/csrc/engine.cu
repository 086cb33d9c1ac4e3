// Node-contraction engine. Every hot-path contraction around one node t of <bra| W |ket> with
// environments on some legs is lowered to the same pipeline of batched GEMMs (ket first):
//
//   T_0     = ket_t permuted to [b_C1][b_C2..b_Cm][q][b_open]         (contracted legs first)
//   T_l     = sum_b T_{l-1}[b][rest] E_Cl[w][a][b]  -> [rest][a_Cl]     l = 1..m, one item per
//             distinct prefix (w_C1..w_Cl) of the TTNO entries (shared between entries)
//   Z[slot] = sum_{groups g of slot} sum_q T_m[prefix_g][q][rest] O_g[p][q]  -> [rest][p]
//             where O_g = sum of c_e * op_e over the entries with that prefix and open-leg
//             value (one combined d x d operator per group)
//   closure: env  E_open[slot][a][b] = sum_rest bra_t[a][rest] Z[slot][b][rest]
//            scalar <bra|H|ket>       = sum bra_t * Z
//            local  (H_eff x)         = Z
//
// This is the contraction order "absorb the ket into the environments leg by leg, apply the
// local operators, close with the bra" of Sec. II.C (Figs. variational and als), with the TTNO
// kept block-sparse: only distinct (w-prefix) and (prefix, w_open) combinations are contracted.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>

#include "internal.h"

namespace {

long long key_of(int node, int open) { return (long long)node * 64 + (open + 1); }

}  // namespace

void StageHost::finalize() {
  n_ua = (long long)std::set<long long>(seg_a.begin(), seg_a.end()).size();
  n_ub = (long long)std::set<long long>(seg_b.begin(), seg_b.end()).size();
  n_seg = (long long)seg_a.size();
  single = true;
  for (size_t j = 0; j + 1 < seg_ptr.size(); ++j) single = single && seg_ptr[j + 1] - seg_ptr[j] == 1;
  a4 = b4 = c2 = c4 = true;
  for (long long a : seg_a) a4 = a4 && a % 4 == 0;
  for (long long b : seg_b) b4 = b4 && b % 4 == 0;
  for (long long c : sub_c) c2 = c2 && c % 2 == 0;
  for (long long c : sub_c) c4 = c4 && c % 4 == 0;
  grp_max = 0;
  for (size_t q = 0; q + 1 < grp_ptr.size(); ++q) grp_max = std::max(grp_max, grp_ptr[q + 1] - grp_ptr[q]);
}

NodePlan& get_plan(ttn_ttno* H, int t, int open) {
  const long long key = key_of(t, open);
  auto it = H->plans.find(key);
  if (it != H->plans.end()) return it->second;
  NodePlan p;
  p.node = t;
  p.open = open;
  const int nl = H->tree.nlegs(t);
  for (int m = 0; m < nl; ++m)
    if (m != open) p.C.push_back(m);
  const int mC = (int)p.C.size();
  p.n_slots = open >= 0 ? H->wdim(t, open) : 1;
  const int d = H->tree.d(t);
  std::vector<std::map<std::vector<int>, int>> pref(mC + 1);
  p.level.resize(mC);
  struct G {
    int prefix, slot;
    std::vector<double> op;
  };
  std::vector<G> groups;
  std::map<std::pair<int, int>, int> gidx;
  struct FG {
    int prefix, slot;
    std::map<int, double> terms;   // w of the last contracted leg -> summed coefficient
  };
  std::vector<FG> fgs;
  std::map<std::pair<int, int>, int> fidx;
  for (const TtnoEntry& e : H->entries[t]) {
    std::vector<int> key;
    int par = 0, par_prev = 0;
    for (int l = 0; l < mC; ++l) {
      key.push_back(e.w[p.C[l]]);
      auto ins = pref[l + 1].emplace(key, (int)pref[l + 1].size());
      if (ins.second) p.level[l].push_back({par, e.w[p.C[l]]});
      par_prev = par;
      par = ins.first->second;
    }
    if (d == 1 && mC >= 1) {
      const int slot_f = open >= 0 ? e.w[open] : 0;
      auto fi = fidx.emplace(std::make_pair(par_prev, slot_f), (int)fgs.size());
      if (fi.second) fgs.push_back({par_prev, slot_f, {}});
      fgs[fi.first->second].terms[e.w[p.C[mC - 1]]] +=
          e.coef * H->op_data[H->op_off[e.op]];
    }
    const int slot = open >= 0 ? e.w[open] : 0;
    auto gi = gidx.emplace(std::make_pair(par, slot), (int)groups.size());
    if (gi.second) groups.push_back({par, slot, std::vector<double>((size_t)d * d, 0.0)});
    std::vector<double>& O = groups[gi.first->second].op;
    const double* src = H->op_data.data() + H->op_off[e.op];
    for (int i = 0; i < d * d; ++i) O[i] += e.coef * src[i];
  }
  std::stable_sort(groups.begin(), groups.end(),
                   [](const G& a, const G& b) { return a.slot < b.slot; });
  p.slot_ptr.assign(p.n_slots + 1, 0);
  for (const G& g : groups) {
    p.grp_prefix.push_back(g.prefix);
    p.slot_ptr[g.slot + 1]++;
    p.ocomb.insert(p.ocomb.end(), g.op.begin(), g.op.end());
  }
  for (int s = 0; s < p.n_slots; ++s) p.slot_ptr[s + 1] += p.slot_ptr[s];
  cudaStream_t st = H->ctx->stream;
  if (d == 1 && mC >= 1) {
    p.fused = true;
    std::stable_sort(fgs.begin(), fgs.end(),
                     [](const FG& a, const FG& b) { return a.slot < b.slot; });
    p.fG_slot_ptr.assign(p.n_slots + 1, 0);
    p.fG_term_ptr.assign(1, 0);
    for (const FG& g : fgs) {
      p.fG_prefix.push_back(g.prefix);
      p.fG_slot_ptr[g.slot + 1]++;
      for (auto& kv : g.terms) {
        p.fT_w.push_back(kv.first);
        p.fT_coef.push_back(kv.second);
      }
      p.fG_term_ptr.push_back((int)p.fT_w.size());
    }
    for (int s2 = 0; s2 < p.n_slots; ++s2) p.fG_slot_ptr[s2 + 1] += p.fG_slot_ptr[s2];
    const size_t nt = std::max<size_t>(p.fT_w.size(), 1);
    p.d_fG_term_ptr = DevBuf(p.fG_term_ptr.size() * sizeof(int), st);
    p.d_fT_w = DevBuf(nt * sizeof(int), st);
    p.d_fT_coef64 = DevBuf(nt * sizeof(double), st);
    p.d_fT_coef32 = DevBuf(nt * sizeof(float), st);
    std::vector<float> c32(p.fT_coef.begin(), p.fT_coef.end());
    CUDA_CHECK(cudaMemcpyAsync(p.d_fG_term_ptr.p, p.fG_term_ptr.data(),
                               p.fG_term_ptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!p.fT_w.empty()) {
      CUDA_CHECK(cudaMemcpyAsync(p.d_fT_w.p, p.fT_w.data(), p.fT_w.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
      CUDA_CHECK(cudaMemcpyAsync(p.d_fT_coef64.p, p.fT_coef.data(),
                                 p.fT_coef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      CUDA_CHECK(cudaMemcpyAsync(p.d_fT_coef32.p, c32.data(), c32.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, st));
    }
    CUDA_CHECK(cudaStreamSynchronize(st));
  }
  const size_t no = std::max<size_t>(p.ocomb.size(), 1);
  p.d_ocomb64 = DevBuf(no * sizeof(double), st);
  p.d_ocomb32 = DevBuf(no * sizeof(float), st);
  std::vector<float> o32(p.ocomb.begin(), p.ocomb.end());
  p.d_slot_ptr = DevBuf(p.slot_ptr.size() * sizeof(int), st);
  p.d_grp_prefix = DevBuf(std::max<size_t>(p.grp_prefix.size(), 1) * sizeof(int), st);
  CUDA_CHECK(cudaMemcpyAsync(p.d_slot_ptr.p, p.slot_ptr.data(), p.slot_ptr.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st));
  if (!p.grp_prefix.empty())
    CUDA_CHECK(cudaMemcpyAsync(p.d_grp_prefix.p, p.grp_prefix.data(),
                               p.grp_prefix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  if (!p.ocomb.empty()) {
    CUDA_CHECK(cudaMemcpyAsync(p.d_ocomb64.p, p.ocomb.data(), p.ocomb.size() * sizeof(double),
                               cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(p.d_ocomb32.p, o32.data(), o32.size() * sizeof(float),
                               cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
  }
  return H->plans.emplace(key, std::move(p)).first->second;
}

namespace {

// Item tables (per stage: C offset per item, CSR of segments with A/B offsets) of one plan for
// concrete bond dimensions; cached in the TTNO.
DevTables& get_tables(ttn_ttno* H, const NodePlan& p, const std::vector<int>& Da,
                      const std::vector<int>& Db, int d, int out_kind,
                      std::vector<long long>& sizes) {
  const int mC = (int)p.C.size();
  const int nl = (int)Da.size();
  sizes.assign(mC + 1, 0);
  long long sz = d;
  for (int m = 0; m < nl; ++m) sz *= Db[m];
  sizes[0] = sz;
  for (int l = 1; l <= mC; ++l) {
    const int c = p.C[l - 1];
    sizes[l] = sizes[l - 1] / Db[c] * Da[c];
  }
  std::vector<long long> key = {p.node, p.open, d, out_kind};
  key.insert(key.end(), Da.begin(), Da.end());
  key.insert(key.end(), Db.begin(), Db.end());
  auto it = H->tables.find(key);
  if (it != H->tables.end()) return it->second;

  using HostStage = StageHost;
  std::vector<HostStage> hs;
  const int n_level_stages = p.fused ? mC - 1 : mC;
  for (int l = 1; l <= n_level_stages; ++l) {
    HostStage s;
    const int c = p.C[l - 1];
    const long long eslice = (long long)Da[c] * Db[c];
    for (size_t j = 0; j < p.level[l - 1].size(); ++j) {
      const auto& pr = p.level[l - 1][j];
      s.seg_a.push_back(l == 1 ? 0 : (long long)pr.first * sizes[l - 1]);
      s.seg_b.push_back((long long)pr.second * eslice);
      s.seg_ptr.push_back((int)s.seg_a.size());
      s.sub_c.push_back((long long)j * sizes[l]);
    }
    hs.push_back(std::move(s));
  }
  if (p.fused) {
    // segmented last level: Z[slot] = sum_{G in slot} T_{m-1}[prefix(G)] x Et[G]
    HostStage s;
    const int c = p.C[mC - 1];
    const long long eslice = (long long)Da[c] * Db[c];
    const long long zsize = sizes[mC];
    for (int slot = 0; slot < p.n_slots; ++slot) {
      for (int G = p.fG_slot_ptr[slot]; G < p.fG_slot_ptr[slot + 1]; ++G) {
        s.seg_a.push_back(mC == 1 ? 0 : (long long)p.fG_prefix[G] * sizes[mC - 1]);
        s.seg_b.push_back((long long)G * eslice);
      }
      s.seg_ptr.push_back((int)s.seg_a.size());
      s.sub_c.push_back((long long)slot * zsize);
    }
    hs.push_back(std::move(s));
  } else {
    HostStage s;
    const long long zsize = sizes[mC];
    for (int slot = 0; slot < p.n_slots; ++slot) {
      for (int g = p.slot_ptr[slot]; g < p.slot_ptr[slot + 1]; ++g) {
        s.seg_a.push_back(mC == 0 ? 0 : (long long)p.grp_prefix[g] * sizes[mC]);
        s.seg_b.push_back((long long)g * d * d);
      }
      s.seg_ptr.push_back((int)s.seg_a.size());
      s.sub_c.push_back((long long)slot * zsize);
    }
    hs.push_back(std::move(s));
  }
  // A groups of the level stages: single-segment items reading the same A slice, in chunks the
  // bulk-copy level kernel stages at once
  for (int l = 1; l <= mC; ++l) {
    HostStage& s = hs[l - 1];
    const int c = p.C[l - 1];
    const int cap = level_group_cap((int)(sizes[l - 1] / Db[c]), Da[c], Db[c]);
    bool single = cap > 0;
    for (size_t j = 0; single && j + 1 < s.seg_ptr.size(); ++j)
      single = s.seg_ptr[j + 1] - s.seg_ptr[j] == 1;
    if (!single) continue;
    std::map<long long, std::vector<int>> by_a;
    for (int j = 0; j + 1 < (int)s.seg_ptr.size(); ++j) by_a[s.seg_a[s.seg_ptr[j]]].push_back(j);
    for (auto& kv : by_a)
      for (size_t i = 0; i < kv.second.size(); i += cap) {
        const size_t e = std::min(kv.second.size(), i + (size_t)cap);
        s.grp_sub.insert(s.grp_sub.end(), kv.second.begin() + i, kv.second.begin() + e);
        s.grp_ptr.push_back((int)s.grp_sub.size());
        s.grp_a.push_back(kv.first);
        for (size_t k = i; k < e; ++k) {
          const int j = kv.second[k];
          s.grp_b.push_back(s.seg_b[s.seg_ptr[j]]);
          s.grp_c.push_back(s.sub_c[j]);
        }
      }
  }
  if (out_kind == OUT_ENV) {
    HostStage s;
    const int o = p.open;
    const long long zsize = sizes[mC];
    for (int slot = 0; slot < p.n_slots; ++slot) {
      s.seg_a.push_back(0);
      s.seg_b.push_back((long long)slot * zsize);
      s.seg_ptr.push_back((int)s.seg_a.size());
      s.sub_c.push_back((long long)slot * Da[o] * Db[o]);
    }
    hs.push_back(std::move(s));
  }
  for (auto& s : hs) s.finalize();
  // pack into one device buffer
  size_t bytes = 0;
  for (auto& s : hs) {
    bytes += (s.sub_c.size() + s.seg_a.size() + s.seg_b.size()) * sizeof(long long);
    bytes += (s.seg_ptr.size() + s.grp_ptr.size() + s.grp_sub.size()) * sizeof(int) +
             (s.grp_a.size() + s.grp_b.size() + s.grp_c.size()) * sizeof(long long) + 10 * 16;
  }
  std::vector<char> host(bytes + 64, 0);
  DevTables t;
  t.buf = DevBuf(bytes + 64, H->ctx->stream);
  size_t off = 0;
  char* dbase = static_cast<char*>(t.buf.p);
  auto put = [&](const void* src, size_t n) -> const void* {
    off = (off + 15) & ~size_t(15);
    if (n) std::memcpy(host.data() + off, src, n);
    const void* dp = dbase + off;
    off += n;
    return dp;
  };
  for (auto& s : hs) {
    StageDev ds;
    ds.n_sub = (int)s.sub_c.size();
    ds.sub_c = (const long long*)put(s.sub_c.data(), s.sub_c.size() * sizeof(long long));
    ds.seg_ptr = (const int*)put(s.seg_ptr.data(), s.seg_ptr.size() * sizeof(int));
    ds.seg_a = (const long long*)put(s.seg_a.data(), s.seg_a.size() * sizeof(long long));
    ds.seg_b = (const long long*)put(s.seg_b.data(), s.seg_b.size() * sizeof(long long));
    ds.n_grp = (int)s.grp_ptr.size() - 1;
    ds.grp_ptr = (const int*)put(s.grp_ptr.data(), s.grp_ptr.size() * sizeof(int));
    ds.grp_sub = (const int*)put(s.grp_sub.data(), s.grp_sub.size() * sizeof(int));
    ds.grp_a = (const long long*)put(s.grp_a.data(), s.grp_a.size() * sizeof(long long));
    ds.grp_b = (const long long*)put(s.grp_b.data(), s.grp_b.size() * sizeof(long long));
    ds.grp_c = (const long long*)put(s.grp_c.data(), s.grp_c.size() * sizeof(long long));
    t.stages.push_back(ds);
  }
  t.host = hs;
  CUDA_CHECK(cudaMemcpyAsync(t.buf.p, host.data(), off, cudaMemcpyHostToDevice, H->ctx->stream));
  CUDA_CHECK(cudaStreamSynchronize(H->ctx->stream));
  return H->tables.emplace(key, std::move(t)).first->second;
}

}  // namespace

template <>
const double* block_node<double>(const ttn_block* b, int t) {
  return b->node64(t);
}
template <>
const float* block_node<float>(const ttn_block* b, int t) {
  return b->node32(t);
}

template <class T>
void node_op(ttn_ctx* ctx, ttn_ttno* H, int t, int open, const ttn_block* bra,
             const ttn_block* ket, const PairSet& ps, const std::vector<const T*>& env,
             const std::vector<int>& env_da, void* out, long long out_len, int out_kind,
             const T* ket_ptr, int ket_n) {
  const int P = ps.P;
  const T* ket_data = ket_ptr ? ket_ptr : block_node<T>(ket, t);
  const int n_ket = ket_ptr ? ket_n : ket->n_states;
  const int* d_pb = ps.d_pb;
  const int* d_pk = ps.d_pk;
  const TreeInfo& tr = H->tree;
  const int nl = tr.nlegs(t), d = tr.d(t);
  NodePlan& p = get_plan(H, t, open);
  const int mC = (int)p.C.size();
  std::vector<int> Da(nl), Db(nl), Dw(nl);
  for (int m = 0; m < nl; ++m) {
    Db[m] = ket->bdim(t, m);
    Dw[m] = H->wdim(t, m);
    Da[m] = bra ? bra->bdim(t, m) : env_da[m];
  }
  std::vector<long long> sizes;
  DevTables& tab = get_tables(H, p, Da, Db, d, out_kind, sizes);
  cudaStream_t st = ctx->stream;

  // The intermediates T_l and Z grow with the number of pairs; beyond the workspace budget
  // (TTN_WORKSPACE_GB, default 24 GB) the pairs are contracted in consecutive chunks, each
  // reading its own slice of the environments and writing its own slice of the output.
  {
    long long per_pair = 0;
    const int n_levels = p.fused ? mC - 1 : mC;
    for (int l = 1; l <= n_levels; ++l) per_pair += (long long)p.level[l - 1].size() * sizes[l];
    if (p.fused && mC >= 1) {
      const int c = p.C[mC - 1];
      per_pair += (long long)p.fG_prefix.size() * Da[c] * Db[c];
    }
    if (out_kind != OUT_LOCAL) per_pair += (long long)p.n_slots * sizes[mC];
    per_pair *= (long long)sizeof(T);
    const char* env_gb = getenv("TTN_WORKSPACE_GB");
    const double budget = (env_gb ? atof(env_gb) : 24.0) * 1e9;
    const long long chunk = std::max<long long>(1, (long long)(budget / std::max<long long>(per_pair, 1)));
    if (P > chunk) {
      long long out_per_pair = 0;
      if (out_kind == OUT_ENV) out_per_pair = (long long)p.n_slots * Da[open] * Db[open];
      else if (out_kind == OUT_LOCAL) out_per_pair = (long long)p.n_slots * sizes[mC];
      else {
        out_per_pair = 1;
      }
      const size_t out_elem = out_kind == OUT_SCALAR ? sizeof(double) : sizeof(T);
      for (long long c0 = 0; c0 < P; c0 += chunk) {
        const int Pc = (int)std::min<long long>(chunk, P - c0);
        PairSet pc{Pc, ps.d_pb + c0, ps.d_pk + c0, ps.max_bra, ps.max_ket};
        std::vector<const T*> envc(env.size(), nullptr);
        for (int m = 0; m < nl; ++m)
          if (env[m]) envc[m] = env[m] + c0 * ((long long)Dw[m] * Da[m] * Db[m]);
        void* outc = static_cast<char*>(out) + (size_t)(c0 * out_per_pair) * out_elem;
        node_op<T>(ctx, H, t, open, bra, ket, pc, envc, env_da, outc,
                   out_len - c0 * out_per_pair, out_kind, ket_ptr, ket_n);
      }
      return;
    }
  }

  // T_0: permuted ket of every ket state
  std::vector<int> kd(Db.begin(), Db.end());
  kd.push_back(d);
  std::vector<int> perm(p.C.begin(), p.C.end());
  perm.push_back(nl);
  if (open >= 0) perm.push_back(open);
  const long long ksize = ket->size[t];
  DevBuf kp((size_t)n_ket * ksize * sizeof(T), st);
  launch_permute<T>(ctx, ket_data, kp.as<T>(), n_ket, nl + 1, kd.data(), perm.data());

  const void* prev = kp.p;
  long long prev_len = (long long)n_ket * ksize;
  int prev_mode = MODE_KET;
  long long prev_pstride = ksize;
  std::vector<DevBuf> Tl(mC + 1);
  const int n_levels = p.fused ? mC - 1 : mC;
  for (int l = 1; l <= n_levels; ++l) {
    const int c = p.C[l - 1];
    const long long rest = sizes[l - 1] / Db[c];
    const int nsub = (int)p.level[l - 1].size();
    Tl[l] = DevBuf((size_t)P * nsub * sizes[l] * sizeof(T), st);
    GemmDesc g{};
    g.M = (int)rest;
    g.N = Da[c];
    g.K = Db[c];
    g.a_sm = 1;
    g.a_sk = rest;
    g.b_sn = Db[c];
    g.b_sk = 1;
    g.c_sm = Da[c];
    g.c_sn = 1;
    g.A = {prev, prev_mode, prev_pstride};
    g.B = {env[c], MODE_PAIR, (long long)Dw[c] * Da[c] * Db[c]};
    g.C = Tl[l].p;
    g.c_mode = MODE_PAIR;
    g.c_pstride = (long long)nsub * sizes[l];
    g.n_pairs = P;
    g.pair_bra = d_pb;
    g.pair_ket = d_pk;
    g.st = tab.stages[l - 1];
    g.hst = &tab.host[l - 1];
    g.a_len = l == 1 ? (long long)n_ket * ksize : prev_len;
    g.b_len = (long long)P * Dw[c] * Da[c] * Db[c];
    g.c_len = (long long)P * g.c_pstride;
    g.max_bra = ps.max_bra;
    g.max_ket = ps.max_ket;
    g.alg_a = l == 1;          // the ket's node tensor (permuted); later levels read T_{l-1}
    g.alg_b = true;            // environment
    g.alg_c = false;           // T_l
    if (level_shape_ok(g)) launch_level<T>(ctx, g);
    else launch_gemm<T>(ctx, g);
    prev_len = g.c_len;
    prev = Tl[l].p;
    prev_mode = MODE_PAIR;
    prev_pstride = g.c_pstride;
  }

  const long long zsize = sizes[mC];
  const long long zrest = zsize / d;
  DevBuf zbuf;
  void* Z = out;
  if (out_kind != OUT_LOCAL) {
    zbuf = DevBuf((size_t)P * p.n_slots * zsize * sizeof(T), st);
    Z = zbuf.p;
  }
  const long long z_len = out_kind == OUT_LOCAL ? out_len : (long long)P * p.n_slots * zsize;
  if (p.fused) {
    // fold the TTNO into the last contracted leg's environment, then one segmented level stage
    const int c = p.C[mC - 1];
    const int nG = (int)p.fG_prefix.size();
    const long long eslice = (long long)Da[c] * Db[c];
    DevBuf Et((size_t)std::max<long long>((long long)P * nG * eslice, 1) * sizeof(T), st);
    int max_w = 0;
    for (int x : p.fT_w) max_w = std::max(max_w, x);
    const void* coef = sizeof(T) == 8 ? p.d_fT_coef64.p : p.d_fT_coef32.p;
    launch_combine_env<T>(ctx, env[c], (long long)Dw[c] * eslice, Da[c], Db[c], Et.as<T>(), P, nG,
                          p.d_fG_term_ptr.as<int>(), p.d_fT_w.as<int>(),
                          static_cast<const T*>(coef), max_w);
    GemmDesc g{};
    const long long rest = sizes[mC - 1] / Db[c];
    g.M = (int)rest;
    g.N = Da[c];
    g.K = Db[c];
    g.a_sm = 1;
    g.a_sk = rest;
    g.b_sn = 1;          // Et slices are stored [b][a]
    g.b_sk = Da[c];
    g.c_sm = Da[c];
    g.c_sn = 1;
    g.A = {prev, prev_mode, prev_pstride};
    g.B = {Et.p, MODE_PAIR, (long long)nG * eslice};
    g.C = Z;
    g.c_mode = MODE_PAIR;
    g.c_pstride = (long long)p.n_slots * zsize;
    g.n_pairs = P;
    g.pair_bra = d_pb;
    g.pair_ket = d_pk;
    g.st = tab.stages[mC - 1];
    g.hst = &tab.host[mC - 1];
    g.a_len = prev_len;
    g.b_len = std::max<long long>((long long)P * nG * eslice, 1);
    g.c_len = z_len;
    g.max_bra = ps.max_bra;
    g.max_ket = ps.max_ket;
    g.alg_a = prev_mode == MODE_KET;
    g.alg_b = false;           // folded environments (their sources count in combine_env)
    g.alg_c = out_kind == OUT_LOCAL;
    if (level_shape_ok(g)) launch_level<T>(ctx, g);
    else launch_gemm<T>(ctx, g);
  } else {
    OpStageDesc o{};
    o.d = d;
    o.rows = (int)zrest;
    o.n_slots = p.n_slots;
    o.n_groups = (int)p.grp_prefix.size();
    o.tsize = zsize;
    o.A = {prev, prev_mode, prev_pstride};
    o.slot_ptr = p.d_slot_ptr.as<int>();
    o.grp_prefix = p.d_grp_prefix.as<int>();
    o.ops = sizeof(T) == 8 ? p.d_ocomb64.p : p.d_ocomb32.p;
    o.Z = Z;
    o.z_pstride = (long long)p.n_slots * zsize;
    o.n_pairs = P;
    o.pair_bra = d_pb;
    o.pair_ket = d_pk;
    o.a_len = prev_len;
    o.z_len = z_len;
    o.max_ket = ps.max_ket;
    o.max_prefix = 0;
    for (int x : p.grp_prefix) o.max_prefix = std::max(o.max_prefix, x);
    o.n_unique_prefix = (int)std::set<int>(p.grp_prefix.begin(), p.grp_prefix.end()).size();
    o.alg_in = prev_mode == MODE_KET;
    o.alg_out = out_kind == OUT_LOCAL;
    launch_op_stage<T>(ctx, o);
  }

  if (out_kind == OUT_ENV) {
    std::vector<int> bd(Da.begin(), Da.end());
    bd.push_back(d);
    std::vector<int> bperm = {open};
    bperm.insert(bperm.end(), p.C.begin(), p.C.end());
    bperm.push_back(nl);
    const long long bsize = bra->size[t];
    DevBuf bp((size_t)bra->n_states * bsize * sizeof(T), st);
    launch_permute<T>(ctx, block_node<T>(bra, t), bp.as<T>(), bra->n_states, nl + 1, bd.data(),
                      bperm.data());
    const long long K = zsize / Db[open];
    GemmDesc g{};
    g.M = Da[open];
    g.N = Db[open];
    g.K = (int)K;
    g.a_sm = K;
    g.a_sk = 1;
    g.b_sn = K;
    g.b_sk = 1;
    g.c_sm = Db[open];
    g.c_sn = 1;
    g.A = {bp.p, MODE_BRA, bsize};
    g.B = {Z, MODE_PAIR, (long long)p.n_slots * zsize};
    g.C = out;
    g.c_mode = MODE_PAIR;
    g.c_pstride = (long long)p.n_slots * Da[open] * Db[open];
    g.n_pairs = P;
    g.pair_bra = d_pb;
    g.pair_ket = d_pk;
    const int cl = p.fused ? mC : mC + 1;   // index of the closure stage in the tables
    g.st = tab.stages[cl];
    g.hst = &tab.host[cl];
    g.a_len = (long long)bra->n_states * bsize;
    g.b_len = (long long)P * p.n_slots * zsize;
    g.c_len = out_len;
    g.max_bra = ps.max_bra;
    g.max_ket = ps.max_ket;
    g.alg_a = true;            // the bra's node tensor (permuted)
    g.alg_b = false;           // Z
    g.alg_c = true;            // the environment
    if (closure_shape_ok(g)) launch_closure<T>(ctx, g);
    else launch_gemm<T>(ctx, g);
  } else if (out_kind == OUT_SCALAR) {
    TTN_REQUIRE(zsize == bra->size[t] && out_len >= P, "scalar closure: shape mismatch");
    launch_pair_dot<T>(ctx, block_node<T>(bra, t), bra->size[t], static_cast<const T*>(Z), zsize,
                       zsize, P, d_pb, static_cast<double*>(out), ps.max_bra,
                       (long long)bra->n_states * bra->size[t], (long long)P * zsize);
  }
}

template <class T>
void envs_compute(ttn_ctx* ctx, ttn_ttno* H, const ttn_block* bra, const ttn_block* ket,
                  const PairSet& ps, int direction, std::vector<DevBuf>& up,
                  std::vector<DevBuf>& down) {
  const int P = ps.P;
  const TreeInfo& tr = H->tree;
  up.resize(tr.n);
  down.resize(tr.n);
  cudaStream_t st = ctx->stream;
  auto esize = [&](int c) {
    return (long long)H->wbond[c] * bra->bond[c] * ket->bond[c];
  };
  for (int t : tr.post) {
    if (t == tr.root) continue;
    const int nl = tr.nlegs(t);
    std::vector<const T*> env(nl, nullptr);
    for (int m = 1; m < nl; ++m) env[m] = up[tr.legs[t][m]].as<T>();
    up[t] = DevBuf((size_t)P * esize(t) * sizeof(T), st);
    node_op<T>(ctx, H, t, 0, bra, ket, ps, env, {}, up[t].p, (long long)P * esize(t), OUT_ENV);
  }
  if (direction == 0) return;
  for (int u : tr.pre) {
    const int nl = tr.nlegs(u);
    const int off = u == tr.root ? 0 : 1;
    for (int m = off; m < nl; ++m) {
      const int c = tr.legs[u][m];
      std::vector<const T*> env(nl, nullptr);
      if (off) env[0] = down[u].as<T>();
      for (int m2 = off; m2 < nl; ++m2)
        if (m2 != m) env[m2] = up[tr.legs[u][m2]].as<T>();
      down[c] = DevBuf((size_t)P * esize(c) * sizeof(T), st);
      node_op<T>(ctx, H, u, m, bra, ket, ps, env, {}, down[c].p, (long long)P * esize(c),
                 OUT_ENV);
    }
  }
}

template void node_op<double>(ttn_ctx*, ttn_ttno*, int, int, const ttn_block*, const ttn_block*,
                              const PairSet&, const std::vector<const double*>&,
                              const std::vector<int>&, void*, long long, int, const double*,
                              int);
template void node_op<float>(ttn_ctx*, ttn_ttno*, int, int, const ttn_block*, const ttn_block*,
                             const PairSet&, const std::vector<const float*>&,
                             const std::vector<int>&, void*, long long, int, const float*, int);
template void envs_compute<double>(ttn_ctx*, ttn_ttno*, const ttn_block*, const ttn_block*,
                                   const PairSet&, int, std::vector<DevBuf>&,
                                   std::vector<DevBuf>&);
template void envs_compute<float>(ttn_ctx*, ttn_ttno*, const ttn_block*, const ttn_block*,
                                  const PairSet&, int, std::vector<DevBuf>&,
                                  std::vector<DevBuf>&);
