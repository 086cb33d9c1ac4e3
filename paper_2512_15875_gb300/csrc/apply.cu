// Exact TTNO x TTNS product (Sec. II.C.1, the direct contraction whose cost Appendix A lists):
//   out[s][(w_0,b_0), (w_1,b_1), ..., p] = sum_q W[w_0, w_1, ..., p, q] in[s][b_0, b_1, ..., q]
// Each merged bond keeps the TTNO index as the major one. W is used block-sparse: one combined
// d x d operator per distinct w-tuple. The kernel is a pure streaming pass (HBM-bound): every
// output element is written once, every input row is read once per w-tuple.
#include <map>

#include "internal.h"

namespace {

struct ApplyArgs {
  int nl, d;
  long long rows;          // prod_m Db_m
  long long in_size, out_size;
  int db[TTN_MAX_LEGS];    // input bond per leg
  long long os[TTN_MAX_LEGS];  // output stride of merged leg m (in elements, p innermost)
};

template <class T>
__global__ void apply_kernel(const T* __restrict__ in, double* __restrict__ out,
                             const long long* __restrict__ grp_off,
                             const T* __restrict__ grp_op, int n_groups, int n_states,
                             ApplyArgs a) {
  const long long per_state = (long long)n_groups * a.rows * a.d;
  const long long total = per_state * n_states;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx / per_state);
    long long r = idx - s * per_state;
    const int g = (int)(r / (a.rows * a.d));
    r -= (long long)g * a.rows * a.d;
    const int p = (int)(r % a.d);
    long long row = r / a.d;
    // output offset of this b-tuple
    long long off = grp_off[g] + p, rr = row;
    for (int m = a.nl - 1; m >= 0; --m) {
      off += (rr % a.db[m]) * a.os[m];
      rr /= a.db[m];
    }
    const T* x = in + (long long)s * a.in_size + row * a.d;
    const T* O = grp_op + ((long long)g * a.d + p) * a.d;
    T acc = T(0);
    for (int q = 0; q < a.d; ++q) acc = fma(O[q], x[q], acc);
    out[(long long)s * a.out_size + off] = (double)acc;
  }
}

}  // namespace

extern "C" ttn_status ttn_apply_block(ttn_ctx* ctx, const ttn_ttno* Hc, const ttn_block* in,
                                      ttn_block** out, ttn_precision prec) {
  if (!ctx || !Hc || !in || !out) return TTN_EINVAL;
  try {
    ttn_ttno* H = const_cast<ttn_ttno*>(Hc);
    TTN_REQUIRE(H->tree.same_shape(in->tree), "TTNO and block live on different trees");
    TTN_REQUIRE(valid_precision(prec), "unknown precision");
    const TreeInfo& tr = in->tree;
    std::vector<int> nb(tr.n);
    for (int i = 0; i < tr.n; ++i) nb[i] = H->wbond[i] * in->bond[i];
    ttn_block* ob = nullptr;
    ttn_status st;
    {
      ttn_tree tmp;
      tmp.ctx = ctx;
      tmp.info = tr;
      st = ttn_block_create(ctx, &tmp, in->n_states, nb.data(), &ob);
      if (st != TTN_OK) return st;
    }
    std::unique_ptr<ttn_block> guard(ob);
    cudaStream_t s = ctx->stream;
    for (int t = 0; t < tr.n; ++t) {
      const int nl = tr.nlegs(t), d = tr.d(t);
      std::map<std::vector<int>, std::vector<double>> groups;
      for (const TtnoEntry& e : H->entries[t]) {
        std::vector<int> w(e.w, e.w + nl);
        auto& O = groups[w];
        if (O.empty()) O.assign((size_t)d * d, 0.0);
        const double* src = H->op_data.data() + H->op_off[e.op];
        for (int i = 0; i < d * d; ++i) O[i] += e.coef * src[i];
      }
      ApplyArgs a{};
      a.nl = nl;
      a.d = d;
      a.rows = 1;
      for (int m = 0; m < nl; ++m) {
        a.db[m] = in->bdim(t, m);
        a.rows *= a.db[m];
      }
      a.in_size = in->size[t];
      a.out_size = ob->size[t];
      long long stride = d;
      for (int m = nl - 1; m >= 0; --m) {
        a.os[m] = stride;
        stride *= ob->bdim(t, m);
      }
      std::vector<long long> goff;
      std::vector<double> gop;
      for (auto& kv : groups) {
        long long off = 0;
        for (int m = 0; m < nl; ++m) off += (long long)kv.first[m] * a.db[m] * a.os[m];
        goff.push_back(off);
        gop.insert(gop.end(), kv.second.begin(), kv.second.end());
      }
      const int ng = (int)goff.size();
      if (ng == 0 || in->n_states == 0) continue;
      DevBuf doff(goff.size() * sizeof(long long), s);
      CUDA_CHECK(cudaMemcpyAsync(doff.p, goff.data(), goff.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice, s));
      const long long total = (long long)ng * a.rows * d * in->n_states;
      const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 64);
      if (prec == TTN_FP64) {
        DevBuf dop(gop.size() * sizeof(double), s);
        CUDA_CHECK(cudaMemcpyAsync(dop.p, gop.data(), gop.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
        LaunchScope ls(ctx, "apply_f64", 2.0 * total * d,
                       8.0 * ((double)in->n_states * a.in_size + total));
        apply_kernel<double><<<blocks, 256, 0, s>>>(in->node64(t), ob->node64(t),
                                                    doff.as<long long>(), dop.as<double>(), ng,
                                                    in->n_states, a);
        CUDA_LAUNCH_CHECK();
        CUDA_CHECK(cudaStreamSynchronize(s));
      } else {
        std::vector<float> g32(gop.begin(), gop.end());
        DevBuf dop(g32.size() * sizeof(float), s);
        CUDA_CHECK(cudaMemcpyAsync(dop.p, g32.data(), g32.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, s));
        LaunchScope ls(ctx, "apply_f32", 2.0 * total * d,
                       4.0 * (double)in->n_states * a.in_size + 8.0 * total);
        apply_kernel<float><<<blocks, 256, 0, s>>>(in->node32(t), ob->node64(t),
                                                   doff.as<long long>(), dop.as<float>(), ng,
                                                   in->n_states, a);
        CUDA_LAUNCH_CHECK();
        CUDA_CHECK(cudaStreamSynchronize(s));
      }
    }
    ob->touch();
    *out = guard.release();
    ctx->last_error.clear();
    return TTN_OK;
  } catch (const TtnError& e) {
    ctx->last_error = e.msg;
    return e.st;
  }
}
