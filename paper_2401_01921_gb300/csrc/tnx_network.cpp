// Network blueprint, contraction-order search, planner and executor.
//
// arXiv 2401.01921, Sec. 8 (Network): a text blueprint of tensor names and
// dummy labels, TOUT (output leg order) and ORDER (binary contraction tree);
// PutUniTensor maps actual legs onto dummy labels; Launch contracts.  Sec. 8.3
// / Sec. 7: the optimal order comes from dynamic programming with cost capping
// (Pfeifer, Haegeman, Verstraete, PRE 90, 033315, 2014) and is reused while the
// bond dimensions stay the same.
//
// A plan turns the tree into a sequence of pairwise steps.  Each step runs
//   1. the integer matching kernel (once, at plan time) -> fused-sector tables,
//   2. the relayout kernel: every block of both operands into its place in the
//      fused operand matrix of its charge group,
//   3. one grouped-GEMM launch over all groups (FP64, FP32, split BF16/FP16, TF32).
// The product of step s is stored as the fused matrices C_g themselves; its
// blocks are strided views into them, read directly by the next relayout.  A
// final relayout writes the canonical blocks of the output in TOUT order.
// All buffers and task tables are allocated at plan time; a launch only
// rewrites the table of base pointers ("slots") and enqueues kernels, so a
// launch (or a whole Lanczos solve) can be captured in one CUDA graph.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <tuple>

#include "tnx_host.h"

#include "tnx_plan.h"

namespace {

typedef unsigned __int128 u128;

}  // namespace

// --------------------------------------------------------------- parsing
namespace {

std::string trim(const std::string& s) {
  size_t a = s.find_first_not_of(" \t\r"), b = s.find_last_not_of(" \t\r");
  return a == std::string::npos ? std::string() : s.substr(a, b - a + 1);
}

bool valid_name(const std::string& s) {
  if (s.empty()) return false;
  for (char c : s)
    if (!(isalnum((unsigned char)c) || c == '_' || c == '-' || c == '.' || c == '\'' || c == '*')) return false;
  return true;
}

std::vector<std::string> split_labels(const std::string& s) {
  std::vector<std::string> out;
  std::string cur;
  for (char c : s) {
    if (c == ',' || c == ';') {
      std::string t = trim(cur);
      if (!t.empty()) out.push_back(t);
      cur.clear();
    } else {
      cur += c;
    }
  }
  std::string t = trim(cur);
  if (!t.empty()) out.push_back(t);
  return out;
}

int parse_tree(const std::string& s, size_t& pos, const std::vector<NetTensor>& ts, std::vector<TreeNode>& nodes) {
  if (pos < s.size() && s[pos] == '(') {
    ++pos;
    int l = parse_tree(s, pos, ts, nodes);
    if (pos >= s.size() || s[pos] != ',') fail(TNX_ERR_NETWORK, "ORDER: expected ','");
    ++pos;
    int r = parse_tree(s, pos, ts, nodes);
    if (pos >= s.size() || s[pos] != ')') fail(TNX_ERR_NETWORK, "ORDER: expected ')'");
    ++pos;
    nodes.push_back(TreeNode{-1, l, r});
    return (int)nodes.size() - 1;
  }
  size_t b = pos;
  while (pos < s.size() && s[pos] != ',' && s[pos] != ')' && s[pos] != '(') ++pos;
  std::string name = s.substr(b, pos - b);
  for (size_t i = 0; i < ts.size(); ++i)
    if (ts[i].name == name) {
      nodes.push_back(TreeNode{(int)i, -1, -1});
      return (int)nodes.size() - 1;
    }
  fail(TNX_ERR_NETWORK, "ORDER names an unknown tensor '" + name + "'");
}

void set_tree_from_string(tnx_network* net, const std::string& order_in) {
  std::string o;
  for (char c : order_in)
    if (!isspace((unsigned char)c)) o += c;
  std::vector<TreeNode> nodes;
  size_t pos = 0;
  int root = parse_tree(o, pos, net->ts, nodes);
  if (pos != o.size()) fail(TNX_ERR_NETWORK, "ORDER: trailing characters");
  std::vector<int> seen(net->ts.size(), 0);
  for (auto& n : nodes)
    if (n.leaf >= 0) seen[n.leaf]++;
  for (int c : seen)
    if (c != 1) fail(TNX_ERR_NETWORK, "ORDER must name every tensor exactly once");
  net->tree = nodes;
  net->root = root;
}

void set_default_tree(tnx_network* net) {
  std::vector<TreeNode> nodes;
  int cur = -1;
  for (size_t i = 0; i < net->ts.size(); ++i) {
    nodes.push_back(TreeNode{(int)i, -1, -1});
    int leaf = (int)nodes.size() - 1;
    if (cur < 0) {
      cur = leaf;
    } else {
      nodes.push_back(TreeNode{-1, cur, leaf});
      cur = (int)nodes.size() - 1;
    }
  }
  net->tree = nodes;
  net->root = cur;
}

std::string tree_string(const tnx_network* net, int node) {
  const TreeNode& n = net->tree[node];
  if (n.leaf >= 0) return net->ts[n.leaf].name;
  return "(" + tree_string(net, n.l) + "," + tree_string(net, n.r) + ")";
}

// ------------------------------------------------------------ order search
u128 mul_sat(u128 a, u128 b) {
  const u128 maxv = ~(u128)0;
  if (a != 0 && b > maxv / a) return maxv;
  return a * b;
}

// DP over subsets with cost capping (Pfeifer et al. 2014).  Cost of a pairwise
// contraction: product of the dimensions of all distinct legs of both operands.
// Ties keep the first split S1 (containing the lowest member) in increasing
// bitmask order.
// ------------------------------------------ block-sparse order search
// Cost of a pairwise contraction counted over charge sectors instead of
// dense dimensions: an operand made of the zero-flux blocks of its legs,
// contracted over the legs K, costs 2 sum_g H_a(-g) H_k(g) H_b(g) flops, where
// H_S(c) is the number of index combinations of the legs S whose signed charges
// add up to c (a convolution of the legs' sector degeneracies), g the charge
// of the contracted legs seen from the left operand, and the left / right free
// legs must carry -g / +g for both operands to be zero-flux.  Intermediates
// are assumed to hold every zero-flux block of their legs.  Subset dynamic
// programming (no capping; at most 12 tensors) minimises the summed cost;
// ties keep the first split, as in the dense search.
namespace {
typedef std::map<std::vector<int32_t>, double> Hist;

struct SymInfo {
  std::vector<int> kinds, zn;
  std::vector<int32_t> add(const std::vector<int32_t>& a, const std::vector<int32_t>& b) const {
    std::vector<int32_t> c(a.size());
    for (size_t i = 0; i < a.size(); ++i) {
      c[i] = a[i] + b[i];
      if (kinds[i] == TNX_ZN) c[i] %= zn[i];
    }
    return c;
  }
  std::vector<int32_t> neg(const std::vector<int32_t>& a) const {
    std::vector<int32_t> c(a.size());
    for (size_t i = 0; i < a.size(); ++i) c[i] = kinds[i] == TNX_ZN ? (zn[i] - a[i]) % zn[i] : -a[i];
    return c;
  }
};

Hist hist_conv(const Hist& a, const Hist& b, const SymInfo& sy) {
  Hist c;
  for (auto& x : a)
    for (auto& y : b) c[sy.add(x.first, y.first)] += x.second * y.second;
  return c;
}

Hist leg_hist(const BondD& b) {
  Hist h;
  for (int s = 0; s < b.nsec; ++s) {
    std::vector<int32_t> q(b.nsym);
    for (int c = 0; c < b.nsym; ++c) q[c] = b.signed_q(s, c);
    h[q] += (double)b.deg[s];
  }
  return h;
}
}  // namespace

void sparse_optimal_tree(tnx_network* net) {
  const int n = (int)net->ts.size();
  if (n > 12) fail(TNX_ERR_UNSUPPORTED, "the block-sparse order search supports at most 12 tensors");
  SymInfo sy;
  const BondD& b0 = net->ts[0].t->bonds[0];
  sy.kinds = b0.kinds;
  sy.zn = b0.zn;
  const int nsym = b0.nsym;
  // label -> (tensor, bond) of each occurrence
  std::map<std::string, std::vector<std::pair<int, const BondD*>>> occ;
  for (int i = 0; i < n; ++i) {
    const NetTensor& t = net->ts[i];
    for (size_t j = 0; j < t.labels.size(); ++j) occ[t.labels[j]].push_back({i, &t.t->bonds[t.perm[j]]});
  }
  std::vector<std::string> labs;
  for (auto& kv : occ) labs.push_back(kv.first);
  const int nl = (int)labs.size();
  std::vector<std::vector<int>> legs(n);
  for (int i = 0; i < n; ++i)
    for (auto& l : net->ts[i].labels) legs[i].push_back((int)(std::find(labs.begin(), labs.end(), l) - labs.begin()));
  const uint32_t full = (1u << n) - 1;
  std::vector<std::vector<int>> open(full + 1);
  std::vector<int> cnt(nl);
  for (uint32_t m = 1; m <= full; ++m) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int i = 0; i < n; ++i)
      if (m >> i & 1)
        for (int l : legs[i]) cnt[l]++;
    for (int l = 0; l < nl; ++l)
      if (cnt[l] == 1) open[m].push_back(l);
  }
  // the bond of label l as it appears inside subset m
  auto bond_in = [&](int l, uint32_t m) -> const BondD& {
    for (auto& o : occ[labs[l]])
      if (m >> o.first & 1) return *o.second;
    fail(TNX_ERR_NETWORK, "internal: label outside its subset");
    return *occ[labs[l]][0].second;
  };
  const Hist unit = {{std::vector<int32_t>(nsym, 0), 1.0}};
  auto hist_of = [&](const std::vector<int>& ls, uint32_t m) {
    Hist h = unit;
    for (int l : ls) h = hist_conv(h, leg_hist(bond_in(l, m)), sy);
    return h;
  };
  auto pair_cost = [&](uint32_t a, uint32_t b) {
    std::vector<int> fa, fb, k;
    for (int l : open[a]) (std::find(open[b].begin(), open[b].end(), l) != open[b].end() ? k : fa).push_back(l);
    for (int l : open[b])
      if (std::find(open[a].begin(), open[a].end(), l) == open[a].end()) fb.push_back(l);
    const Hist ha = hist_of(fa, a), hk = hist_of(k, a), hb = hist_of(fb, b);
    double c = 0.0;
    for (auto& g : hk) {
      auto ia = ha.find(sy.neg(g.first));
      auto ib = hb.find(g.first);
      if (ia != ha.end() && ib != hb.end()) c += 2.0 * ia->second * g.second * ib->second;
    }
    return c;
  };
  std::vector<double> best(full + 1, 0.0);
  std::vector<uint32_t> split(full + 1, 0);
  for (int size = 2; size <= n; ++size)
    for (uint32_t m = 1; m <= full; ++m) {
      if (__builtin_popcount(m) != size) continue;
      uint32_t low = m & (~m + 1), rest = m ^ low, s = 0;
      bool found = false;
      double bc = 0.0;
      while (true) {
        uint32_t m1 = low | s, m2 = m ^ m1;
        if (m2 != 0) {
          const double c = best[m1] + best[m2] + pair_cost(m1, m2);
          if (!found || c < bc) {
            found = true;
            bc = c;
            split[m] = m1;
          }
        }
        if (s == rest) break;
        s = (s - rest) & rest;
      }
      best[m] = bc;
    }
  std::vector<TreeNode> nodes;
  std::function<int(uint32_t)> build = [&](uint32_t m) -> int {
    if (__builtin_popcount(m) == 1) {
      nodes.push_back(TreeNode{__builtin_ctz(m), -1, -1});
      return (int)nodes.size() - 1;
    }
    int l = build(split[m]);
    int r = build(m ^ split[m]);
    nodes.push_back(TreeNode{-1, l, r});
    return (int)nodes.size() - 1;
  };
  int root = build(full);
  net->tree = nodes;
  net->root = root;
}

void optimal_tree(tnx_network* net) {
  const int n = (int)net->ts.size();
  if (n > 20) fail(TNX_ERR_UNSUPPORTED, "optimal order search supports at most 20 tensors");
  std::map<std::string, int64_t> dims;
  for (auto& t : net->ts)
    for (size_t j = 0; j < t.labels.size(); ++j) dims[t.labels[j]] = t.t->bonds[t.perm[j]].dim;
  std::vector<std::string> labs;
  for (auto& kv : dims) labs.push_back(kv.first);
  const int nl = (int)labs.size();
  std::vector<std::vector<int>> legs(n);
  for (int i = 0; i < n; ++i)
    for (auto& l : net->ts[i].labels) legs[i].push_back((int)(std::find(labs.begin(), labs.end(), l) - labs.begin()));
  const uint32_t full = (1u << n) - 1;
  // open legs of each subset: legs appearing exactly once inside it
  std::vector<std::vector<int>> open(full + 1);
  std::vector<int> cnt(nl);
  for (uint32_t m = 1; m <= full; ++m) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int i = 0; i < n; ++i)
      if (m >> i & 1)
        for (int l : legs[i]) cnt[l]++;
    for (int l = 0; l < nl; ++l)
      if (cnt[l] == 1) open[m].push_back(l);
  }
  std::vector<int> mark(nl, 0);
  auto pair_cost = [&](uint32_t a, uint32_t b) {
    u128 c = 1;
    for (int l : open[a]) { mark[l] = 1; c = mul_sat(c, (u128)dims[labs[l]]); }
    for (int l : open[b])
      if (!mark[l]) c = mul_sat(c, (u128)dims[labs[l]]);
    for (int l : open[a]) mark[l] = 0;
    return c;
  };
  u128 mu = 1;
  for (int i = 0; i < n; ++i) {
    u128 s = 1;
    for (int l : legs[i]) s = mul_sat(s, (u128)dims[labs[l]]);
    if (s > mu) mu = s;
  }
  const u128 INF = ~(u128)0;
  std::vector<u128> best(full + 1);
  std::vector<uint32_t> split(full + 1);
  std::vector<char> have(full + 1);
  std::vector<int> order_by_size;
  std::vector<uint32_t> masks;
  for (int size = 2; size <= n; ++size)
    for (uint32_t m = 1; m <= full; ++m)
      if (__builtin_popcount(m) == size) masks.push_back(m);
  while (true) {
    std::fill(have.begin(), have.end(), 0);
    for (int i = 0; i < n; ++i) { best[1u << i] = 0; have[1u << i] = 1; }
    u128 rejected = INF;
    for (uint32_t m : masks) {
      uint32_t low = m & (~m + 1), rest = m ^ low;
      bool found = false;
      u128 bc = 0;
      uint32_t bs = 0;
      uint32_t s = 0;
      while (true) {
        uint32_t m1 = low | s, m2 = m ^ m1;
        if (m2 != 0 && have[m1] && have[m2]) {
          u128 c = best[m1] + best[m2];
          u128 pc = pair_cost(m1, m2);
          c = (c + pc < c) ? INF : c + pc;
          if (c > mu) {
            if (c < rejected) rejected = c;
          } else if (!found || c < bc) {
            found = true;
            bc = c;
            bs = m1;
          }
        }
        if (s == rest) break;
        s = (s - rest) & rest;
      }
      if (found) { best[m] = bc; split[m] = bs; have[m] = 1; }
    }
    if (have[full]) break;
    u128 nm = mul_sat(mu, 2);
    mu = rejected > nm ? rejected : nm;
  }
  std::vector<TreeNode> nodes;
  std::function<int(uint32_t)> build = [&](uint32_t m) -> int {
    if (__builtin_popcount(m) == 1) {
      nodes.push_back(TreeNode{__builtin_ctz(m), -1, -1});
      return (int)nodes.size() - 1;
    }
    int l = build(split[m]);
    int r = build(m ^ split[m]);
    nodes.push_back(TreeNode{-1, l, r});
    return (int)nodes.size() - 1;
  };
  int root = build(full);
  net->tree = nodes;
  net->root = root;
}

// ------------------------------------------------------------------ views
std::vector<int64_t> rowmajor(const int64_t* shape, int r) {
  std::vector<int64_t> s(r);
  int64_t acc = 1;
  for (int l = r - 1; l >= 0; --l) { s[l] = acc; acc *= shape[l]; }
  return s;
}

void sort_view(OpView& v) {
  const int r = v.rank();
  std::vector<int64_t> idx(v.nblk);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return std::lexicographical_compare(v.qn.begin() + a * r, v.qn.begin() + (a + 1) * r, v.qn.begin() + b * r,
                                        v.qn.begin() + (b + 1) * r);
  });
  std::vector<int32_t> qn(v.qn.size());
  std::vector<int64_t> base(v.nblk), stride(v.stride.size());
  std::vector<int64_t> rs(v.rowstart.size()), rl(v.rowld.size());
  for (int64_t i = 0; i < v.nblk; ++i) {
    std::copy(v.qn.begin() + idx[i] * r, v.qn.begin() + (idx[i] + 1) * r, qn.begin() + i * r);
    std::copy(v.stride.begin() + idx[i] * r, v.stride.begin() + (idx[i] + 1) * r, stride.begin() + i * r);
    base[i] = v.base[idx[i]];
    if (!rs.empty()) {
      rs[i] = v.rowstart[idx[i]];
      rl[i] = v.rowld[idx[i]];
    }
  }
  v.qn.swap(qn);
  v.base.swap(base);
  v.stride.swap(stride);
  v.rowstart.swap(rs);
  v.rowld.swap(rl);
}

OpView input_view(const NetTensor& nt, int slot) {
  const tnx_tensor* t = nt.t;
  const int r = t->rank;
  OpView v;
  v.slot = slot;
  v.labels = nt.labels;
  for (int j = 0; j < r; ++j) v.bonds.push_back(t->bonds[nt.perm[j]]);
  v.nblk = t->nblk;
  v.qn.resize((size_t)v.nblk * r);
  v.stride.resize((size_t)v.nblk * r);
  v.base = t->off;
  for (int64_t b = 0; b < t->nblk; ++b) {
    auto st = rowmajor(&t->shape[(size_t)b * r], r);
    for (int j = 0; j < r; ++j) {
      v.qn[(size_t)b * r + j] = t->qn[(size_t)b * r + nt.perm[j]];
      v.stride[(size_t)b * r + j] = st[nt.perm[j]];
    }
  }
  sort_view(v);
  return v;
}

// Drop unit legs and merge neighbours that are contiguous in both source and destination.
// Division by the invariant d for indices n < 2^31 (Granlund and Montgomery,
// PLDI 1994): with p = ceil(log2 d) and m = ceil(2^(31+p) / d), m < 2^32 and
// floor(n / d) = floor(n m / 2^(31+p)) = umulhi(n, m) >> (p - 1), because
// n m / 2^(31+p) exceeds n / d by less than 1 / d.  d = 1: magic 0 (q = n).
void leg_magic(uint64_t d, uint32_t& magic, uint8_t& shift) {
  magic = 0;
  shift = 0;
  if (d > 1) {
    int lg = 0;
    while ((1ull << lg) < d) ++lg;
    magic = (uint32_t)(((1ull << (31 + lg)) + d - 1) / d);
    shift = (uint8_t)(lg - 1);
  }
}

void finish_task(CopyTask& t, std::vector<int64_t> shape, std::vector<int64_t> ss, std::vector<int64_t> ds) {
  std::vector<int64_t> sh2, s2, d2;
  for (size_t l = 0; l < shape.size(); ++l) {
    if (shape[l] == 1) continue;
    if (!sh2.empty() && s2.back() == ss[l] * shape[l] && d2.back() == ds[l] * shape[l]) {
      sh2.back() *= shape[l];
      s2.back() = ss[l];
      d2.back() = ds[l];
    } else {
      sh2.push_back(shape[l]);
      s2.push_back(ss[l]);
      d2.push_back(ds[l]);
    }
  }
  if (sh2.empty()) { sh2.push_back(1); s2.push_back(1); d2.push_back(1); }
  if (sh2.size() > TNX_MAXR) fail(TNX_ERR_UNSUPPORTED, "block copy of rank above the limit");
  t.rank = (int)sh2.size();
  t.nelem = 1;
  int64_t smax = 0, dmax = 0;
  for (size_t l = 0; l < sh2.size(); ++l) {
    if (sh2[l] > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "block extent above 2^31");
    smax += (sh2[l] - 1) * s2[l];
    dmax += (sh2[l] - 1) * d2[l];
    t.nelem *= sh2[l];
  }
  if (t.nelem > INT32_MAX || smax > INT32_MAX || dmax > INT32_MAX)
    fail(TNX_ERR_UNSUPPORTED, "block relayout with element offsets above 2^31");
  for (int l = 0; l < TNX_MAXR; ++l) {
    t.shape[l] = 1;
    t.magic[l] = 0;
    t.shift[l] = 0;
    t.sstride[l] = t.dstride[l] = 0;
  }
  for (size_t l = 0; l < sh2.size(); ++l) {
    const uint64_t d = (uint64_t)sh2[l];
    t.shape[l] = (int32_t)d;
    t.sstride[l] = (int32_t)s2[l];
    t.dstride[l] = (int32_t)d2[l];
    leg_magic(d, t.magic[l], t.shift[l]);
  }
  // transposing task: the source's unit-stride leg is not the destination's
  // (small blocks stay plain tasks: a 32 x 32 tile per CTA would mostly idle,
  // while packed with their neighbours they share one CTA)
  t.tleg = -1;
  if (t.src_slot >= 0 && t.rank >= 2 && t.nelem >= 256) {
    int S = -1;
    for (int l = 0; l < t.rank; ++l)
      if (t.sstride[l] == 1 && t.shape[l] > 1) S = l;
    if (S >= 0 && S != t.rank - 1 && t.shape[S] >= 8 && t.dstride[t.rank - 1] == 1) t.tleg = S;
  }
}

// A block copy before it is finished: its legs in task order, and where its
// rows lie in a row-major matrix on either side, when that is known (the
// packed GEMM operands on the destination side, GEMM outputs on the source
// side).
struct RawTask {
  CopyTask t;                          // slots and base offsets
  std::vector<int64_t> shape, ss, ds;
  std::vector<char> drow, srow;        // leg is a row leg of the destination / source matrix
  int64_t drow0 = -1, dW = 0;          // destination: offset of the block's first row start; row length
  int64_t srow0 = -1, sW = 0;          // source: the same
};

// A band member's legs (P, Q, I): extent, wide-side stride, narrow-side stride.
struct BandLegs {
  int64_t ext[3], wst[3], nst[3];
  int64_t wcol;
};

// Views a block as a band member on the wide side `dside` (destination or
// source): at most two row legs (P outer, Q inner) and one column leg I that is
// contiguous on the wide side, after extent-1 legs are dropped and legs
// contiguous on both sides are merged.  False when the block does not fit.
bool band_legs(const RawTask& r, bool dside, BandLegs& b) {
  const std::vector<int64_t>& ws = dside ? r.ds : r.ss;
  const std::vector<int64_t>& nsv = dside ? r.ss : r.ds;
  const std::vector<char>& isrow = dside ? r.drow : r.srow;
  struct Leg { int64_t e, w, n; };
  std::vector<Leg> rows, cols;
  for (size_t l = 0; l < r.shape.size(); ++l) {
    if (r.shape[l] == 1) continue;
    (isrow[l] ? rows : cols).push_back(Leg{r.shape[l], ws[l], nsv[l]});
  }
  auto reduce = [](std::vector<Leg>& v) {
    std::sort(v.begin(), v.end(), [](const Leg& a, const Leg& b) { return a.w > b.w; });
    std::vector<Leg> o;
    for (const Leg& g : v) {
      if (!o.empty() && o.back().w == g.w * g.e && o.back().n == g.n * g.e) {
        o.back().e *= g.e;
        o.back().w = g.w;
        o.back().n = g.n;
      } else {
        o.push_back(g);
      }
    }
    v.swap(o);
  };
  reduce(rows);
  reduce(cols);
  if (rows.size() > 2 || cols.size() > 1) return false;
  const Leg one{1, 0, 0};
  const Leg P = rows.size() == 2 ? rows[0] : one;
  const Leg Q = rows.size() == 2 ? rows[1] : (rows.size() == 1 ? rows[0] : one);
  const Leg I = cols.empty() ? one : cols[0];
  if (!cols.empty() && I.w != 1) return false;
  const Leg L3[3] = {P, Q, I};
  for (int k = 0; k < 3; ++k) {
    b.ext[k] = L3[k].e;
    b.wst[k] = L3[k].w;
    b.nst[k] = L3[k].n;
  }
  b.wcol = dside ? r.t.dst_off - r.drow0 : r.t.src_off - r.srow0;
  const int64_t W = dside ? r.dW : r.sW;
  return b.wcol >= 0 && b.wcol + I.e <= W;
}

// Turns the raw copies into tasks: blocks that share the rows of a narrow
// matrix (<= 96 columns) on the destination side, else on the source side,
// become bands; everything else is finished as a plain task.  A destination
// band writes whole rows, so it must hold every block written into those
// rows: rows with a block that does not fit are left to plain tasks.  Bands
// serve the fused skinny step only (on their own they measured no faster than
// plain tasks, and far slower for many small blocks): destination bands with
// `dest_bands` (the operand such a step gathers), source bands with
// `source_first` (the output of such a step, which it stores straight into
// this operand when the operand is made of source bands only).
std::vector<CopyTask> emit_tasks(const std::vector<RawTask>& raw, bool dest_bands, bool source_first) {
  constexpr int64_t kMaxW = 96;
  std::vector<CopyTask> out;
  std::vector<char> used(raw.size(), 0);
  for (int pass = 0; pass < 2; ++pass) {
    const bool dside = source_first ? pass == 1 : pass == 0;
    typedef std::tuple<int, int64_t, int64_t> Key;   // slot, first row start, row length
    std::map<Key, std::vector<std::pair<size_t, BandLegs>>> bands;
    std::set<Key> bad;
    for (size_t i = 0; i < raw.size(); ++i) {
      const RawTask& r = raw[i];
      const int64_t row0 = dside ? r.drow0 : r.srow0, W = dside ? r.dW : r.sW;
      const int slot = dside ? r.t.dst_slot : r.t.src_slot;
      if (row0 < 0 || slot < 0) continue;
      const Key k(slot, row0, W);
      // a block already moved by a source band still writes into these
      // destination rows: they cannot be written whole
      if (used[i]) {
        if (dside) bad.insert(k);
        continue;
      }
      BandLegs b;
      if (W > kMaxW || !band_legs(r, dside, b)) bad.insert(k);
      else bands[k].push_back({i, b});
    }
    for (auto& kv : bands) {
      if (bad.count(kv.first)) continue;
      auto& m = kv.second;
      const int64_t W = std::get<2>(kv.first);
      const BandLegs& f = m[0].second;
      bool ok = m.size() <= TNX_BAND_MAXM, narrow = false;
      for (auto& x : m) {
        const BandLegs& b = x.second;
        for (int k = 0; k < 2; ++k) ok = ok && b.ext[k] == f.ext[k] && (b.ext[k] == 1 || b.wst[k] == f.wst[k]);
        narrow = narrow || b.ext[2] < 16;
      }
      const int64_t EP = f.ext[0], EQ = f.ext[1], Wp = W | 1;
      // rows of a row-major matrix: (p, q) starts at row0 + (p * EQ + q) * W
      ok = ok && (EQ == 1 || f.wst[1] == W) && (EP == 1 || f.wst[0] == EQ * W) && EP * EQ * W <= INT32_MAX;
      for (auto& x : m) {
        const BandLegs& b = x.second;
        int64_t nmax = 0;
        for (int k = 0; k < 3; ++k) nmax += (b.ext[k] - 1) * b.nst[k];
        ok = ok && nmax <= INT32_MAX;
      }
      if (!ok || (dside ? !dest_bands : !(source_first && narrow))) continue;
      // tile: up to 64 rows along the leg the members' narrow sides run along
      const bool qin = EQ > 1 && (EP == 1 || f.nst[1] <= f.nst[0]);
      const int64_t Ein = qin ? EQ : EP, Eout = qin ? EP : EQ;
      // balanced: the tiles of a leg differ in extent by one at most
      auto balance = [](int64_t E, int64_t Tmax) {
        const int64_t n = (E + Tmax - 1) / Tmax;
        return (E + n - 1) / n;
      };
      const int64_t Tin = balance(Ein, std::min<int64_t>(64, std::max<int64_t>(1, TNX_BAND_CAP / Wp)));
      const int64_t Tout = balance(Eout, std::max<int64_t>(1, TNX_BAND_CAP / (Tin * Wp)));
      CopyTask h;
      memset(&h, 0, sizeof(h));
      h.tleg = TNX_BAND_HEADER;
      h.rank = (int)m.size();
      h.src_slot = dside ? -1 : std::get<0>(kv.first);
      h.dst_slot = dside ? std::get<0>(kv.first) : -1;
      (dside ? h.dst_off : h.src_off) = std::get<1>(kv.first);
      h.shape[0] = (int32_t)EP;
      h.shape[1] = (int32_t)EQ;
      h.shape[2] = (int32_t)W;
      h.shape[3] = (int32_t)(qin ? Tout : Tin);
      h.shape[4] = (int32_t)(qin ? Tin : Tout);
      h.shape[5] = dside ? 1 : 0;
      h.shape[6] = qin ? 1 : 0;
      h.sstride[0] = (int32_t)(EP > 1 ? f.wst[0] : 0);
      h.sstride[1] = (int32_t)(EQ > 1 ? f.wst[1] : 0);
      out.push_back(h);
      for (auto& x : m) {
        const RawTask& r = raw[x.first];
        const BandLegs& b = x.second;
        CopyTask t = r.t;
        t.rank = 3;
        t.nelem = b.ext[0] * b.ext[1] * b.ext[2];
        for (int k = 0; k < TNX_MAXR; ++k) {
          t.shape[k] = 1;
          t.sstride[k] = t.dstride[k] = 0;
          t.magic[k] = 0;
          t.shift[k] = 0;
        }
        for (int k = 0; k < 3; ++k) {
          t.shape[k] = (int32_t)b.ext[k];
          t.sstride[k] = (int32_t)(dside ? b.nst[k] : b.wst[k]);
          t.dstride[k] = (int32_t)(dside ? b.wst[k] : b.nst[k]);
          leg_magic((uint64_t)b.ext[k], t.magic[k], t.shift[k]);
        }
        t.tleg = TNX_BAND_MEMBER;
        t.wcol = (int32_t)b.wcol;
        out.push_back(t);
        used[x.first] = 1;
      }
    }
  }
  for (size_t i = 0; i < raw.size(); ++i) {
    if (used[i]) continue;
    CopyTask t = raw[i].t;
    finish_task(t, raw[i].shape, raw[i].ss, raw[i].ds);
    out.push_back(t);
  }
  return out;
}

}  // namespace

// The same copies as plain tasks: band headers dropped, members finished as
// ordinary tasks (a destination band's row gaps are zeros already).
std::vector<CopyTask> tnx_unband_tasks(const std::vector<CopyTask>& tasks) {
  std::vector<CopyTask> out;
  for (const CopyTask& t : tasks) {
    if (t.tleg == TNX_BAND_HEADER) continue;
    if (t.tleg != TNX_BAND_MEMBER) {
      out.push_back(t);
      continue;
    }
    CopyTask u = t;
    std::vector<int64_t> shape, ss, ds;
    for (int l = 0; l < t.rank; ++l) {
      shape.push_back(t.shape[l]);
      ss.push_back(t.sstride[l]);
      ds.push_back(t.dstride[l]);
    }
    u.wcol = 0;
    finish_task(u, shape, ss, ds);
    out.push_back(u);
  }
  return out;
}

// Chunks of the relayout kernel (see k_copy.cu): large tasks cut into pieces of
// TNX_COPY_CHUNK elements, consecutive small tasks packed together, transposing
// tasks cut into 32 x 32 tiles, bands into their tiles.
void tnx_make_copy_chunks(const std::vector<CopyTask>& tasks, std::vector<int4>& chunks) {
  chunks.clear();
  size_t i = 0;
  while (i < tasks.size()) {
    const CopyTask& t = tasks[i];
    if (t.nelem > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "block above 2^31 elements");
    if (t.tleg == TNX_BAND_MEMBER) fail(TNX_ERR_ARG, "internal: band member without its header");
    if (t.tleg == TNX_BAND_HEADER) {
      const int64_t ntiles = (int64_t)((t.shape[0] + t.shape[3] - 1) / t.shape[3]) *
                             ((t.shape[1] + t.shape[4] - 1) / t.shape[4]);
      for (int64_t k = 0; k < ntiles; ++k) chunks.push_back(make_int4((int)i, (int)k, -2, 0));
      i += 1 + (size_t)t.rank;
    } else if (t.tleg >= 0) {
      const int64_t ncols = t.shape[t.tleg], nrows = t.nelem / ncols;
      const int64_t ntiles = ((nrows + 31) / 32) * ((ncols + 31) / 32);
      for (int64_t k = 0; k < ntiles; ++k) chunks.push_back(make_int4((int)i, (int)k, -1, 0));
      ++i;
    } else if (t.nelem >= TNX_COPY_CHUNK / 2) {
      for (int64_t e = 0; e < t.nelem; e += TNX_COPY_CHUNK)
        chunks.push_back(make_int4((int)i, (int)e, 1, (int)std::min<int64_t>(TNX_COPY_CHUNK, t.nelem - e)));
      ++i;
    } else {
      size_t j = i;
      int64_t tot = 0;
      while (j < tasks.size() && j - i < TNX_COPY_PACK && tasks[j].tleg == -1 && tasks[j].nelem < TNX_COPY_CHUNK / 2 &&
             tot + tasks[j].nelem <= TNX_COPY_CHUNK)
        tot += tasks[j++].nelem;
      chunks.push_back(make_int4((int)i, 0, (int)(j - i), (int)tot));
      i = j;
    }
  }
  if (chunks.size() > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "too many relayout chunks");
}

namespace {

// Every element a task touches must lie inside its slot's buffer: checked on
// the host before anything is launched.
void validate_tasks(const Plan& p, const std::vector<CopyTask>& tasks) {
  for (size_t i = 0; i < tasks.size(); ++i) {
    const CopyTask& t = tasks[i];
    if (t.tleg == TNX_BAND_HEADER) {
      // the tile fits the staging buffer, the members follow, and the wide rows
      // (p, q, c), c < W, lie inside the wide slot
      const int EP = t.shape[0], EQ = t.shape[1], W = t.shape[2], TP = t.shape[3], TQ = t.shape[4];
      const bool dw = t.shape[5] != 0;
      const int slot = dw ? t.dst_slot : t.src_slot;
      const int64_t base = dw ? t.dst_off : t.src_off;
      if (t.rank < 1 || t.rank > TNX_BAND_MAXM || i + t.rank >= tasks.size() || EP < 1 || EQ < 1 || W < 1 ||
          TP < 1 || TQ < 1 || TP > EP || TQ > EQ || (int64_t)TP * TQ * (W | 1) > TNX_BAND_CAP ||
          t.sstride[0] < 0 || t.sstride[1] < 0)
        fail(TNX_ERR_ARG, "internal: malformed relayout band");
      const int64_t mw = base + (int64_t)(EP - 1) * t.sstride[0] + (int64_t)(EQ - 1) * t.sstride[1] + W - 1;
      if (slot < 0 || slot >= (int)p.slot_elems.size() || base < 0 || mw >= p.slot_elems[slot])
        fail(TNX_ERR_ARG, "internal: relayout band out of bounds");
      std::vector<std::pair<int, int>> cols;
      for (int k = 1; k <= t.rank; ++k) cols.push_back({tasks[i + k].wcol, tasks[i + k].shape[2]});
      std::sort(cols.begin(), cols.end());
      for (size_t k = 1; k < cols.size(); ++k)
        if (cols[k - 1].first + cols[k - 1].second > cols[k].first) fail(TNX_ERR_ARG, "internal: overlapping band members");
      for (int k = 1; k <= t.rank; ++k) {
        const CopyTask& m = tasks[i + k];
        const int32_t* ws = dw ? m.dstride : m.sstride;
        if (m.tleg != TNX_BAND_MEMBER || m.rank != 3 || m.shape[0] != EP || m.shape[1] != EQ || m.wcol < 0 ||
            (int64_t)m.wcol + m.shape[2] > W || (dw ? m.dst_slot : m.src_slot) != slot ||
            (dw ? m.dst_off : m.src_off) != base + m.wcol || (EP > 1 && ws[0] != t.sstride[0]) ||
            (EQ > 1 && ws[1] != t.sstride[1]) || (m.shape[2] > 1 && ws[2] != 1))
          fail(TNX_ERR_ARG, "internal: malformed relayout band member");
      }
      continue;
    }
    int64_t ms = t.src_off, md = t.dst_off;
    for (int l = 0; l < t.rank; ++l) {
      if (t.sstride[l] < 0 || t.dstride[l] < 0 || t.shape[l] < 1) fail(TNX_ERR_ARG, "internal: malformed relayout task");
      ms += (int64_t)(t.shape[l] - 1) * t.sstride[l];
      md += (int64_t)(t.shape[l] - 1) * t.dstride[l];
    }
    if (t.dst_slot < 0 || t.dst_slot >= (int)p.slot_elems.size() || t.dst_off < 0 || md >= p.slot_elems[t.dst_slot])
      fail(TNX_ERR_ARG, "internal: relayout destination out of bounds");
    if (t.src_slot >= 0 && (t.src_slot >= (int)p.slot_elems.size() || t.src_off < 0 || ms >= p.slot_elems[t.src_slot]))
      fail(TNX_ERR_ARG, "internal: relayout source out of bounds");
  }
}

TaskList upload_tasks(Plan& p, const std::vector<CopyTask>& tasks) {
  validate_tasks(p, tasks);
  TaskList tl;
  std::vector<int4> chunks;
  tl.total = 0;
  tnx_make_copy_chunks(tasks, chunks);
  for (size_t i = 0; i < tasks.size(); ++i) tl.total += tasks[i].nelem;
  if (chunks.size() > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "too many relayout chunks");
  tl.n = (int)tasks.size();
  tl.nchunks = (int)chunks.size();
  tl.d = p.upload(tasks);
  tl.chunks = p.upload(chunks);
  tl.h = tasks;
  tl.hchunks = chunks;
  return tl;
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------ matching (device)
void run_match(Plan& p, StepPlan& s) {
  tnx_ctx* ctx = p.ctx;
  const OpView &A = s.A, &B = s.B;
  MatchArgs a;
  memset(&a, 0, sizeof(a));
  const int nsym = A.rank() ? A.bonds[0].nsym : (B.rank() ? B.bonds[0].nsym : 0);
  s.nsym = nsym;
  a.nk = (int)s.ka.size();
  a.nfa = (int)s.fa.size();
  a.nfb = (int)s.fb.size();
  a.nsym = nsym;
  if (a.nk > TNX_MAXR || a.nfa > TNX_MAXR || a.nfb > TNX_MAXR) fail(TNX_ERR_UNSUPPORTED, "rank above the limit");
  std::vector<int64_t> deg;
  std::vector<int32_t> kq;
  auto add_leg = [&](const BondD& b, MatchLeg& ml, bool kleg) {
    ml.nsec = b.nsec;
    ml.sec_base = (int)deg.size();
    for (int sct = 0; sct < b.nsec; ++sct) {
      deg.push_back(b.deg[sct]);
      for (int c = 0; c < nsym; ++c) kq.push_back(kleg ? b.signed_q(sct, c) : 0);
    }
  };
  int64_t kspace = 1, faspace = 1, fbspace = 1;
  for (int i = 0; i < a.nk; ++i) { add_leg(A.bonds[s.ka[i]], a.kleg[i], true); kspace *= A.bonds[s.ka[i]].nsec; }
  for (int i = 0; i < a.nfa; ++i) { add_leg(A.bonds[s.fa[i]], a.faleg[i], false); faspace *= A.bonds[s.fa[i]].nsec; }
  for (int i = 0; i < a.nfb; ++i) { add_leg(B.bonds[s.fb[i]], a.fbleg[i], false); fbspace *= B.bonds[s.fb[i]].nsec; }
  const int64_t LIM = int64_t(1) << 26;
  if (kspace > LIM || faspace > LIM || fbspace > LIM) fail(TNX_ERR_UNSUPPORTED, "sector tuple space above 2^26");
  int64_t cspace = 1;
  for (int c = 0; c < nsym; ++c) {
    const BondD& b0 = A.bonds[0];
    a.zn[c] = b0.kinds[c] == TNX_ZN ? b0.zn[c] : 0;
    if (a.zn[c] > 0) {
      a.clo[c] = 0;
      a.crange[c] = a.zn[c];
    } else {
      int64_t lo = 0, hi = 0;
      for (int i = 0; i < a.nk; ++i) {
        const BondD& b = A.bonds[s.ka[i]];
        int32_t mn = INT32_MAX, mx = INT32_MIN;
        for (int sct = 0; sct < b.nsec; ++sct) { mn = std::min(mn, b.signed_q(sct, c)); mx = std::max(mx, b.signed_q(sct, c)); }
        lo += mn;
        hi += mx;
      }
      if (hi - lo + 1 > (1 << 22)) fail(TNX_ERR_UNSUPPORTED, "charge range too wide");
      a.clo[c] = (int32_t)lo;
      a.crange[c] = (int32_t)(hi - lo + 1);
    }
    cspace *= a.crange[c];
    if (cspace > (int64_t(1) << 24)) fail(TNX_ERR_UNSUPPORTED, "charge space above 2^24");
  }
  a.kspace = kspace;
  a.faspace = faspace;
  a.fbspace = fbspace;
  a.cspace = cspace;
  a.gmax = (int32_t)std::min<int64_t>(std::min(cspace, kspace), 4096);
  a.nA = A.nblk;
  a.nB = B.nblk;
  a.rA = A.rank();
  a.rB = B.rank();
  for (int i = 0; i < a.nk; ++i) { a.kposA[i] = s.ka[i]; a.kposB[i] = s.kb[i]; }
  for (int i = 0; i < a.nfa; ++i) a.fposA[i] = s.fa[i];
  for (int i = 0; i < a.nfb; ++i) a.fposB[i] = s.fb[i];

  // One device buffer for the call: the results first (one download), then
  // the inputs (one upload), then the kernel's scratch; the kernel clears its
  // scratch itself, so only the two status words are zeroed.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + std::max<size_t>(bytes, 8) + 255) & ~size_t(255);
    return o;
  };
  const size_t o_ng = take(8);
  const size_t o_ch = take((size_t)a.gmax * std::max(nsym, 1) * 4);
  const size_t o_mkn = take((size_t)a.gmax * 3 * 8);
  const size_t o_am = take((size_t)std::max<int64_t>(A.nblk, 1) * 3 * 8);
  const size_t o_bm = take((size_t)std::max<int64_t>(B.nblk, 1) * 3 * 8);
  const size_t out_bytes = off;
  const size_t o_deg = take(deg.size() * 8);
  const size_t o_kq = take(kq.size() * 4);
  const size_t o_qa = take(A.qn.size() * 4);
  const size_t o_qb = take(B.qn.size() * 4);
  const size_t in_end = off;
  const size_t o_kpres = take(kspace * 4), o_kgroup = take(kspace * 4), o_koff = take(kspace * 8);
  const size_t o_rgroup = take(faspace * 4), o_roff = take(faspace * 8);
  const size_t o_cgroup = take(fbspace * 4), o_coff = take(fbspace * 8);
  const size_t o_cspres = take(cspace * 4), o_csgid = take(cspace * 4);
  const size_t o_scan = take(((size_t)1024 * a.gmax + 3 * (size_t)a.gmax) * 8);
  DevBuf buf(ctx, off);
  char* d = (char*)buf.p;
  std::vector<char> hin(in_end - out_bytes, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (bytes) memcpy(hin.data() + (o - out_bytes), src, bytes);
  };
  put(o_deg, deg.data(), deg.size() * 8);
  put(o_kq, kq.data(), kq.size() * 4);
  put(o_qa, A.qn.data(), A.qn.size() * 4);
  put(o_qb, B.qn.data(), B.qn.size() * 4);
  CUDA_CHECK(cudaMemcpyAsync(d + out_bytes, hin.data(), hin.size(), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_CHECK(cudaMemsetAsync(d + o_ng, 0, 8, ctx->stream));
  a.deg = (const int64_t*)(d + o_deg);
  a.kcharge = (const int32_t*)(d + o_kq);
  a.qA = (const int32_t*)(d + o_qa);
  a.qB = (const int32_t*)(d + o_qb);
  a.kpres = (int32_t*)(d + o_kpres);
  a.kgroup = (int32_t*)(d + o_kgroup);
  a.koff = (int64_t*)(d + o_koff);
  a.rgroup = (int32_t*)(d + o_rgroup);
  a.roff = (int64_t*)(d + o_roff);
  a.cgroup = (int32_t*)(d + o_cgroup);
  a.coff = (int64_t*)(d + o_coff);
  a.cspres = (int32_t*)(d + o_cspres);
  a.csgid = (int32_t*)(d + o_csgid);
  a.scan_tmp = (int64_t*)(d + o_scan);
  a.ngroups = (int32_t*)(d + o_ng);
  a.status = a.ngroups + 1;
  a.charges = (int32_t*)(d + o_ch);
  a.mkn = (int64_t*)(d + o_mkn);
  a.amap = (int64_t*)(d + o_am);
  a.bmap = (int64_t*)(d + o_bm);
  CUDA_CHECK(tnx_launch_match(a, ctx->stream));
  std::vector<char> hout(out_bytes);
  CUDA_CHECK(cudaMemcpyAsync(hout.data(), d, out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  int32_t hs[2];
  memcpy(hs, hout.data() + o_ng, 8);
  if (hs[1] == 1) fail(TNX_ERR_UNSUPPORTED, "more charge groups than the matching kernel supports");
  if (hs[1] == 2) fail(TNX_ERR_ARG, "internal: charge outside the planned range");
  if (hs[1] == 3) fail(TNX_ERR_ARG, "internal: a block's sector index lies outside its leg");
  s.G = hs[0];
  if (s.G < 0 || s.G > a.gmax) fail(TNX_ERR_ARG, "internal: charge group count out of range");
  s.charges.resize((size_t)s.G * nsym);
  s.mkn.resize((size_t)s.G * 3);
  s.amap.resize((size_t)A.nblk * 3);
  s.bmap.resize((size_t)B.nblk * 3);
  if (s.G && nsym) memcpy(s.charges.data(), hout.data() + o_ch, s.charges.size() * 4);
  if (s.G) memcpy(s.mkn.data(), hout.data() + o_mkn, s.mkn.size() * 8);
  if (A.nblk) memcpy(s.amap.data(), hout.data() + o_am, s.amap.size() * 8);
  if (B.nblk) memcpy(s.bmap.data(), hout.data() + o_bm, s.bmap.size() * 8);
}

int64_t block_dim(const OpView& v, int64_t b, const std::vector<int>& legs) {
  int64_t d = 1;
  for (int l : legs) d *= v.bonds[l].deg[v.qn[(size_t)b * v.rank() + l]];
  return d;
}

// ------------------------------------------------------------- step plan
void build_step(Plan& p, StepPlan& s) {
  const OpView &A = s.A, &B = s.B;
  std::vector<std::pair<int, int>> pairs;
  for (int i = 0; i < A.rank(); ++i)
    for (int j = 0; j < B.rank(); ++j)
      if (A.labels[i] == B.labels[j]) pairs.push_back({i, j});
  std::sort(pairs.begin(), pairs.end());
  for (auto& pr : pairs) {
    check_contractible(A.bonds[pr.first], B.bonds[pr.second], A.labels[pr.first]);
    s.ka.push_back(pr.first);
    s.kb.push_back(pr.second);
  }
  for (int i = 0; i < A.rank(); ++i)
    if (std::find(s.ka.begin(), s.ka.end(), i) == s.ka.end()) s.fa.push_back(i);
  for (int j = 0; j < B.rank(); ++j)
    if (std::find(s.kb.begin(), s.kb.end(), j) == s.kb.end()) s.fb.push_back(j);
  if (A.rank() && B.rank() && !A.bonds[0].same_syms(B.bonds[0]))
    fail(TNX_ERR_BOND_MISMATCH, "tensors with different symmetries in one network");

  run_match(p, s);
  const int G = s.G;

  // packed operand layouts: A_g [M x ldK] and B_g [N x ldK] (K-major), C_g [M x N]
  s.ldK.resize(G);
  s.offA.resize(G);
  s.offB.resize(G);
  s.offC.resize(G);
  int64_t oa = 0, ob = 0, oc = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t M = s.mkn[3 * g], K = s.mkn[3 * g + 1], N = s.mkn[3 * g + 2];
    s.ldK[g] = align_up(std::max<int64_t>(K, 1), 4);
    s.offA[g] = oa;
    s.offB[g] = ob;
    s.offC[g] = oc;
    oa = align_up(oa + M * s.ldK[g], 32);
    ob = align_up(ob + N * s.ldK[g], 32);
    oc = align_up(oc + M * N, 32);
  }
  s.slotA = p.new_slot(p.alloc_zero((size_t)oa * 8), oa);
  s.slotB = p.new_slot(p.alloc_zero((size_t)ob * 8), ob);
  s.slotC = p.new_slot(p.alloc_zero((size_t)oc * 8), oc);

  const int rA = A.rank(), rB = B.rank();
  // relayout tasks: block b of operand v (free legs f, contracted legs k) into
  // rows [row, row + rows of b) and columns [col, col + columns of b) of its
  // group's packed matrix (row length ldK)
  auto raw_tasks = [&](const OpView& v, int dst_slot, const std::vector<int64_t>& off, const std::vector<int64_t>& map,
                       int rowi, int coli, const std::vector<int>& f, const std::vector<int>& k, bool dest_bands) {
    std::vector<RawTask> raw;
    const int r = v.rank();
    for (int64_t b = 0; b < v.nblk; ++b) {
      const int64_t g = map[3 * b];
      if (g < 0) continue;
      RawTask x;
      CopyTask& t = x.t;
      memset(&t, 0, sizeof(t));
      t.src_slot = v.slot;
      t.dst_slot = dst_slot;
      t.src_off = v.base[b];
      x.drow0 = off[g] + map[3 * b + rowi] * s.ldK[g];
      x.dW = s.ldK[g];
      t.dst_off = x.drow0 + map[3 * b + coli];
      if (v.nrow >= 0) {
        x.srow0 = v.rowstart[b];
        x.sW = v.rowld[b];
      }
      for (int pass = 0; pass < 2; ++pass)
        for (int l : pass ? k : f) {
          x.shape.push_back(v.bonds[l].deg[v.qn[b * r + l]]);
          x.ss.push_back(v.stride[b * r + l]);
          x.drow.push_back(pass == 0);
          x.srow.push_back(l < v.nrow);
        }
      x.ds.assign(x.shape.size(), 0);
      int64_t acc = 1;
      for (int i = (int)x.shape.size() - 1; i >= (int)f.size(); --i) { x.ds[i] = acc; acc *= x.shape[i]; }
      acc = s.ldK[g];
      for (int i = (int)f.size() - 1; i >= 0; --i) { x.ds[i] = acc; acc *= x.shape[i]; }
      raw.push_back(std::move(x));
    }
    return emit_tasks(raw, dest_bands, v.skinny_out && !dest_bands);
  };
  // a step whose groups all have K <= 16 runs on the fused skinny kernel,
  // which gathers its A through destination bands
  bool skinny_step = G > 0;
  for (int g = 0; g < G; ++g) skinny_step = skinny_step && s.mkn[3 * g + 1] <= 16 && s.mkn[3 * g + 2] <= 64;
  s.copyA = upload_tasks(p, raw_tasks(A, s.slotA, s.offA, s.amap, 1, 2, s.fa, s.ka, skinny_step));
  s.copyB = upload_tasks(p, raw_tasks(B, s.slotB, s.offB, s.bmap, 2, 1, s.fb, s.kb, false));

  // grouped GEMM
  std::vector<GemmGroup> gg(G);
  std::vector<GemmTile> tiles, stiles;
  s.skinny.assign(G, 0);
  // Groups with K <= 16 run on the skinny FP64 kernel.  Under split precision
  // that holds only when every group of the step is that small: otherwise the
  // few small groups ride along in the split GEMM launch (one K tile each)
  // instead of costing a launch of their own.
  bool all_small = true;
  for (int g = 0; g < G; ++g) all_small = all_small && s.mkn[3 * g + 1] <= 16;
  const bool split_prec = p.prec == TNX_PREC_SPLIT_BF16 || p.prec == TNX_PREC_SPLIT_F16;
  for (int g = 0; g < G; ++g) {
    GemmGroup& x = gg[g];
    memset(&x, 0, sizeof(x));
    x.a_slot = s.slotA;
    x.b_slot = s.slotB;
    x.c_slot = s.slotC;
    x.a_off = s.offA[g];
    x.b_off = s.offB[g];
    x.c_off = s.offC[g];
    x.M = (int32_t)s.mkn[3 * g];
    x.K = (int32_t)s.mkn[3 * g + 1];
    x.N = (int32_t)s.mkn[3 * g + 2];
    x.lda = x.ldb = (int32_t)s.ldK[g];
    x.ldc = x.N;
    if (x.K <= 16 && (!split_prec || all_small)) {
      s.skinny[g] = 1;
      for (int m0 = 0; m0 < x.M; m0 += 128)
        for (int n0 = 0; n0 < x.N; n0 += 64) stiles.push_back(GemmTile{g, m0, n0, 0});
    } else {
      for (int m0 = 0; m0 < x.M; m0 += 64)
        for (int n0 = 0; n0 < x.N; n0 += 64) tiles.push_back(GemmTile{g, m0, n0, 0});
    }
  }
  s.dG = p.upload(gg);
  s.dT = p.upload(tiles);
  s.ntiles = (int)tiles.size();
  s.dTs = p.upload(stiles);
  s.nstiles_skinny = (int)stiles.size();
  s.hG = gg;
  s.hT = tiles;
  s.hTs = stiles;

  // useful flops: matched block pairs share (group, K offset)
  std::map<std::pair<int64_t, int64_t>, std::pair<double, double>> acc;
  std::map<std::pair<int64_t, int64_t>, double> kd;
  for (int64_t b = 0; b < A.nblk; ++b) {
    if (s.amap[3 * b] < 0) continue;
    auto key = std::make_pair(s.amap[3 * b], s.amap[3 * b + 2]);
    acc[key].first += (double)block_dim(A, b, s.fa);
    kd[key] = (double)block_dim(A, b, s.ka);
  }
  for (int64_t b = 0; b < B.nblk; ++b) {
    if (s.bmap[3 * b] < 0) continue;
    acc[std::make_pair(s.bmap[3 * b], s.bmap[3 * b + 1])].second += (double)block_dim(B, b, s.fb);
  }
  s.flops = 0;
  s.flops_skinny = 0;
  for (auto& kv : acc) {
    const double f = 2.0 * kv.second.first * kd[kv.first] * kv.second.second;
    s.flops += f;
    if (s.skinny[kv.first.first]) s.flops_skinny += f;
  }

  // output view: the fused matrices C_g, one block per (row tuple, column tuple)
  OpView& C = s.C;
  C.slot = s.slotC;
  C.nrow = (int)s.fa.size();
  C.skinny_out = skinny_step;
  for (int l : s.fa) { C.bonds.push_back(A.bonds[l]); C.labels.push_back(A.labels[l]); }
  for (int l : s.fb) { C.bonds.push_back(B.bonds[l]); C.labels.push_back(B.labels[l]); }
  std::vector<std::map<std::vector<int32_t>, int64_t>> rows(G), cols(G);
  for (int64_t b = 0; b < A.nblk; ++b) {
    const int64_t g = s.amap[3 * b];
    if (g < 0) continue;
    std::vector<int32_t> key;
    for (int l : s.fa) key.push_back(A.qn[b * rA + l]);
    rows[g][key] = s.amap[3 * b + 1];
  }
  for (int64_t b = 0; b < B.nblk; ++b) {
    const int64_t g = s.bmap[3 * b];
    if (g < 0) continue;
    std::vector<int32_t> key;
    for (int l : s.fb) key.push_back(B.qn[b * rB + l]);
    cols[g][key] = s.bmap[3 * b + 2];
  }
  const int rC = C.rank();
  for (int g = 0; g < G; ++g) {
    const int64_t N = s.mkn[3 * g + 2];
    for (auto& rr : rows[g])
      for (auto& cc : cols[g]) {
        C.qn.insert(C.qn.end(), rr.first.begin(), rr.first.end());
        C.qn.insert(C.qn.end(), cc.first.begin(), cc.first.end());
        C.base.push_back(s.offC[g] + rr.second * N + cc.second);
        C.rowstart.push_back(s.offC[g] + rr.second * N);
        C.rowld.push_back(N);
        std::vector<int64_t> st(rC);
        int64_t a2 = 1;
        for (int i = (int)cc.first.size() - 1; i >= 0; --i) {
          st[s.fa.size() + i] = a2;
          a2 *= C.bonds[s.fa.size() + i].deg[cc.first[i]];
        }
        a2 = N;
        for (int i = (int)rr.first.size() - 1; i >= 0; --i) {
          st[i] = a2;
          a2 *= C.bonds[i].deg[rr.first[i]];
        }
        C.stride.insert(C.stride.end(), st.begin(), st.end());
        C.nblk++;
      }
  }
  sort_view(C);
}

// final relayout: root view -> canonical output blocks in TOUT order
void build_final(Plan& p, const OpView& root, const std::vector<std::string>& tout) {
  const int r = (int)tout.size();
  if (r != root.rank()) fail(TNX_ERR_NETWORK, "TOUT does not match the open legs");
  std::vector<int> pos(r);
  p.out_bonds.clear();
  for (int j = 0; j < r; ++j) {
    auto it = std::find(root.labels.begin(), root.labels.end(), tout[j]);
    if (it == root.labels.end()) fail(TNX_ERR_NETWORK, "TOUT label '" + tout[j] + "' is not an open leg");
    pos[j] = (int)(it - root.labels.begin());
    p.out_bonds.push_back(root.bonds[pos[j]]);
  }
  p.out_labels = tout;
  std::map<std::vector<int32_t>, int64_t> rootblk;
  for (int64_t b = 0; b < root.nblk; ++b) {
    std::vector<int32_t> k(r);
    for (int j = 0; j < r; ++j) k[j] = root.qn[b * r + pos[j]];
    rootblk[k] = b;
  }
  std::vector<int32_t> qn;
  int64_t nblk;
  enumerate_blocks(p.out_bonds, qn, nblk);
  std::vector<CopyTask> tasks;
  int64_t off = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    std::vector<int32_t> k(qn.begin() + b * r, qn.begin() + (b + 1) * r);
    std::vector<int64_t> shape(r);
    for (int j = 0; j < r; ++j) shape[j] = p.out_bonds[j].deg[k[j]];
    auto ds = rowmajor(shape.data(), r);
    CopyTask t;
    memset(&t, 0, sizeof(t));
    t.dst_slot = p.out_slot;
    t.dst_off = off;
    std::vector<int64_t> ss(r, 0);
    auto it = rootblk.find(k);
    if (it != rootblk.end()) {
      t.src_slot = root.slot;
      t.src_off = root.base[it->second];
      for (int j = 0; j < r; ++j) ss[j] = root.stride[it->second * r + pos[j]];
    } else {
      t.src_slot = -1;
    }
    finish_task(t, shape, ss, ds);
    tasks.push_back(t);
    int64_t n = 1;
    for (auto x : shape) n *= x;
    off += n;
  }
  p.fin = upload_tasks(p, tasks);
}

// The output relayout folded into the last product: when that product runs
// entirely on the split (or TF32) GEMM and every column of each of its charge
// groups lands, over the group's rows r, at out[off + r * stride] (the usual
// case: the GEMM's rows are one leg of the output, e.g. a' of psi'), the GEMM's
// epilogue stores there through a per-column table and the relayout launch is
// skipped.  The table is derived from the relayout's own tasks, element by
// element, and checked: every column is either absent from the output or
// present for all of its group's rows, with one consistent stride.
void fold_final(Plan& p) {
  if (p.steps.empty() || p.fin.h.empty()) return;
  StepPlan& s = p.steps.back();
  const bool split = p.prec == TNX_PREC_SPLIT_BF16 || p.prec == TNX_PREC_SPLIT_F16 || p.prec == TNX_PREC_TF32;
  if (!split || s.nstiles == 0 || s.nstiles_skinny != 0 || s.nftiles != 0 || s.hSG.empty()) return;
  const int G = s.G;
  std::vector<int64_t> fbase(G + 1, 0);
  std::vector<std::pair<int64_t, int>> starts;   // (C offset, group)
  for (int g = 0; g < G; ++g) {
    if (s.skinny[g]) return;
    fbase[g + 1] = fbase[g] + s.mkn[3 * g + 2];
    if (s.mkn[3 * g] > 0 && s.mkn[3 * g + 2] > 0) starts.push_back({s.offC[g], g});
  }
  std::sort(starts.begin(), starts.end());
  const int64_t ncol = fbase[G];
  std::vector<int64_t> r0(ncol, -1), d0(ncol, 0), st(ncol, INT64_MIN), cnt(ncol, 0);
  for (const CopyTask& t : p.fin.h) {
    if (t.src_slot != s.slotC || t.dst_slot != p.out_slot || t.tleg < -1) return;
    std::vector<int64_t> idx(t.rank, 0);
    for (int64_t e = 0; e < t.nelem; ++e) {
      int64_t so = t.src_off, dd = t.dst_off;
      for (int l = 0; l < t.rank; ++l) {
        so += idx[l] * t.sstride[l];
        dd += idx[l] * t.dstride[l];
      }
      for (int l = t.rank - 1; l >= 0; --l) {   // next index, last leg fastest
        if (++idx[l] < t.shape[l]) break;
        idx[l] = 0;
      }
      auto it = std::upper_bound(starts.begin(), starts.end(), std::make_pair(so, INT32_MAX));
      if (it == starts.begin()) return;
      const int g = (--it)->second;
      const int64_t M = s.mkn[3 * g], N = s.mkn[3 * g + 2], rel = so - s.offC[g];
      if (rel >= M * N) return;
      const int64_t r = rel / N, k = fbase[g] + rel % N;
      if (r0[k] < 0) {
        r0[k] = r;
        d0[k] = dd;
      } else {
        const int64_t dr = r - r0[k], dv = dd - d0[k];
        if (dr == 0) return;
        if (st[k] == INT64_MIN) {
          if (dv % dr != 0) return;
          st[k] = dv / dr;
        } else if (dv != st[k] * dr) {
          return;
        }
      }
      ++cnt[k];
    }
  }
  std::vector<FinalCol> fc(std::max<int64_t>(ncol, 1));
  const int64_t out_elems = p.slot_elems[p.out_slot];
  for (int g = 0; g < G; ++g) {
    const int64_t M = s.mkn[3 * g];
    for (int64_t k = fbase[g]; k < fbase[g + 1]; ++k) {
      if (cnt[k] == 0) {
        fc[k] = FinalCol{-1, 0};
        continue;
      }
      if (cnt[k] != M) return;
      const int64_t stride = st[k] == INT64_MIN ? 0 : st[k];
      const int64_t off = d0[k] - r0[k] * stride, last = off + (M - 1) * stride;
      if (off < 0 || off >= out_elems || last < 0 || last >= out_elems) return;
      fc[k] = FinalCol{off, stride};
    }
  }
  const int fslot = p.new_slot((double*)p.upload(fc), (int64_t)fc.size() * 2);
  std::vector<SplitGroup> sg = s.hSG;   // the host copy stays unfolded (batches keep their relayout)
  for (int g = 0; g < G; ++g) {
    sg[g].out_slot = p.out_slot;
    sg[g].fc_slot = fslot;
    sg[g].fc_off = (int32_t)fbase[g];
  }
  s.dSG = p.upload(sg);
  s.split_fold = true;
  p.fin_folded = true;
}

// Fuses every step whose charge groups are all skinny (K <= 16, N <= 64) and
// whose operand A is relaid entirely by destination bands: one kernel gathers
// each band's A rows from their sources, forms the product and writes the
// output rows.  When the step that consumes this step's output relays it
// entirely by source bands over the same rows, the output rows go straight
// into that step's packed operand and its relayout is skipped.  The bands'
// members become per-column descriptors (k_fused.cu).  A consumer that is
// itself fused gathers its A from this output, so it must be written: that
// holds by construction, as a fused step's A relayout is made of destination
// bands, which a scattering step requires to be source bands.
bool fuse_skinny_step(Plan& p, size_t si, int ti, bool tA) {
  {
    StepPlan& s = p.steps[si];
    if (s.nstiles_skinny == 0 || s.ntiles != 0 || s.nstiles != 0) return false;
    bool ok = true;
    int64_t maxld = 1, maxN = 1;
    for (int g = 0; g < s.G; ++g) {
      ok = ok && s.skinny[g];
      maxld = std::max(maxld, s.ldK[g]);
      maxN = std::max(maxN, s.mkn[3 * g + 2]);
    }
    if (!ok || maxld > 16 || maxN > 64) return false;
    // destination bands of A: header, group, first row of the block, extents
    struct Band { size_t h; int g; int64_t row; int EP, EQ; };
    std::vector<Band> bands;
    const std::vector<CopyTask>& ta = s.copyA.h;
    for (size_t i = 0; ok && i < ta.size(); i += 1 + (size_t)ta[i].rank) {
      const CopyTask& h = ta[i];
      if (h.tleg != TNX_BAND_HEADER || h.shape[5] != 1) {
        ok = false;
        break;
      }
      const auto it = std::upper_bound(s.offA.begin(), s.offA.end(), h.dst_off);
      const int g = (int)(it - s.offA.begin()) - 1;
      if (g < 0 || (h.dst_off - s.offA[g]) % s.ldK[g] != 0 || h.shape[2] != s.ldK[g]) {
        ok = false;
        break;
      }
      bands.push_back(Band{i, g, (h.dst_off - s.offA[g]) / s.ldK[g], h.shape[0], h.shape[1]});
    }
    if (!ok || bands.empty()) return false;
    // the consumer of C (step ti): its relayout of C must be source bands only
    std::map<int64_t, size_t> scat;   // C row start -> header
    const std::vector<CopyTask>* tl = nullptr;
    if (ti >= 0) {
      tl = tA ? &p.steps[ti].copyA.h : &p.steps[ti].copyB.h;
      for (size_t i = 0; i < tl->size(); i += 1 + (size_t)(*tl)[i].rank) {
        const CopyTask& h = (*tl)[i];
        if (h.tleg != TNX_BAND_HEADER || h.shape[5] != 0 || h.src_slot != s.slotC) {
          ti = -1;
          break;
        }
        scat[h.src_off] = i;
      }
    }
    std::vector<long long> sidx(bands.size(), -1);   // scatter header, -1: no reader
    if (ti >= 0) {
      size_t matched = 0;
      for (size_t b = 0; b < bands.size() && ti >= 0; ++b) {
        const Band& B = bands[b];
        const auto it = scat.find(s.offC[B.g] + B.row * s.mkn[3 * B.g + 2]);
        if (it == scat.end()) continue;
        const CopyTask& h = (*tl)[it->second];
        if (h.shape[0] != B.EP || h.shape[1] != B.EQ || h.shape[2] != s.mkn[3 * B.g + 2]) ti = -1;
        sidx[b] = (long long)it->second;
        ++matched;
      }
      if (ti >= 0 && matched != scat.size()) ti = -1;
    }
    // column descriptors: a band's members, column by column, with the plan
    // buffers resolved (a fused step touches no rebindable slot)
    std::vector<FusedCol> cols;
    auto internal = [&](int slot) { return slot >= p.nin && slot != p.out_slot && slot < (int)p.h_slots.size(); };
    auto add_cols = [&](const std::vector<CopyTask>& tasks, size_t h, int64_t W, bool gather) {
      const size_t first = cols.size();
      cols.resize(first + (size_t)W, FusedCol{nullptr, 0, 0});
      if (h == (size_t)-1) return first;
      for (int k = 1; k <= tasks[h].rank; ++k) {
        const CopyTask& m = tasks[h + k];
        const int32_t* st = gather ? m.sstride : m.dstride;
        const int slot = gather ? m.src_slot : m.dst_slot;
        if (!internal(slot)) ok = false;
        if (!ok) break;
        for (int i = 0; i < m.shape[2]; ++i) {
          FusedCol& d = cols[first + (size_t)m.wcol + (size_t)i];
          d.ptr = p.h_slots[slot] + (gather ? m.src_off : m.dst_off) + (int64_t)i * st[2];
          d.sP = st[0];
          d.sQ = st[1];
        }
      }
      return first;
    };
    auto balance = [](int64_t E, int64_t Tmax) {
      const int64_t n = (E + Tmax - 1) / Tmax;
      return (E + n - 1) / n;
    };
    std::vector<FusedTile> tiles;
    for (size_t b = 0; b < bands.size(); ++b) {
      const Band& B = bands[b];
      const int64_t N = s.mkn[3 * B.g + 2];
      const size_t gcol = add_cols(ta, B.h, s.ldK[B.g], true);
      int64_t scol = -(int64_t)B.EQ - 1;   // write the rows to C
      if (ti >= 0) scol = (int64_t)add_cols(*tl, sidx[b] < 0 ? (size_t)-1 : (size_t)sidx[b], N, false);
      const int tQ = (int)balance(B.EQ, 16), tP = (int)balance(B.EP, TNX_FUSED_ROWS / tQ);
      for (int p0 = 0; p0 < B.EP; p0 += tP)
        for (int q0 = 0; q0 < B.EQ; q0 += tQ)
          tiles.push_back(FusedTile{B.g, (int32_t)gcol, (int32_t)scol, (int32_t)B.row, p0, q0,
                                    std::min(tP, B.EP - p0), std::min(tQ, B.EQ - q0), (int32_t)s.ldK[B.g],
                                    (int32_t)N, 0, 0});
    }
    // many nearly empty tiles (small sectors) run faster unfused: plain
    // relayouts pack small blocks, the skinny kernel fills 128-row tiles
    int64_t rows = 0;
    for (const Band& B : bands) rows += (int64_t)B.EP * B.EQ;
    if (!ok || tiles.size() > INT32_MAX || cols.size() > INT32_MAX || rows < 32 * (int64_t)tiles.size()) return false;
    s.hFT = tiles;
    s.hFC = cols;
    s.dFT = p.upload(tiles);
    s.dFC = p.upload(cols);
    s.nftiles = (int)tiles.size();
    s.fkp = (int)(maxld | 1);
    s.fnp = (int)(maxN | 1);
    if (ti >= 0) {
      s.fscatter = true;
      StepPlan& t = p.steps[ti];
      (tA ? t.skipA : t.skipB) = true;
    }
  }
  return true;
}

void fuse_skinny_steps(Plan& p) {
  // a relayout whose bands no fused step uses goes back to plain tasks (a
  // relayout holds destination bands, for its own step's gather, or source
  // bands, for the producing step's scatter, never both)
  auto plain = [&](TaskList& t, int dest) {
    for (const CopyTask& x : t.h)
      if (x.tleg == TNX_BAND_HEADER && x.shape[5] == dest) {
        t = upload_tasks(p, tnx_unband_tasks(t.h));
        return;
      }
  };
  auto consumer = [&](size_t si, bool& tA) -> int {
    for (size_t tj = si + 1; tj < p.steps.size(); ++tj) {
      if (p.steps[tj].A.slot == p.steps[si].slotC) return tA = true, (int)tj;
      if (p.steps[tj].B.slot == p.steps[si].slotC) return tA = false, (int)tj;
    }
    return -1;
  };
  for (size_t si = 0; si < p.steps.size(); ++si) {
    StepPlan& s = p.steps[si];
    bool cA = false;
    const int ci = consumer(si, cA);
    const bool fused = fuse_skinny_step(p, si, ci, cA);
    if (!fused) plain(s.copyA, 1);
    if (ci >= 0 && !s.fscatter) plain(cA ? p.steps[ci].copyA : p.steps[ci].copyB, 0);
  }
}

std::string plan_key(const tnx_network* net, const std::string& order) {
  std::string k = order + "#" + std::to_string(net->prec) + (net->narrow_tiles ? "#n" : "#w");
  for (auto& t : net->ts) {
    k += "#" + t.name + "(";
    for (size_t j = 0; j < t.perm.size(); ++j) k += t.t->bonds[t.perm[j]].key() + "/";
    k += ")";
  }
  return k;
}

std::string dims_key(const tnx_network* net) {
  std::string k;
  for (auto& t : net->ts) {
    for (size_t j = 0; j < t.perm.size(); ++j) k += std::to_string(t.t->bonds[t.perm[j]].dim) + ",";
    k += ";";
  }
  return k;
}

void require_put(const tnx_network* net) {
  for (auto& t : net->ts)
    if (!t.t) fail(TNX_ERR_NETWORK, "tensor '" + t.name + "' has not been put");
}

void ensure_order(tnx_network* net) {
  require_put(net);
  if (net->optimal) {
    // the sparse search depends on the sectors, not only the dimensions
    std::string dk = std::to_string(net->optimal) + ":" + dims_key(net);
    if (net->optimal == 2)
      for (auto& t : net->ts)
        for (auto& b : t.t->bonds) dk += b.key();
    if (dk != net->order_dims_key) {
      if (net->optimal == 2) sparse_optimal_tree(net);
      else optimal_tree(net);
      net->order_dims_key = dk;
    }
  }
}

void build_split_parts(Plan& p, StepPlan& s);

// Builds the plan of the network's current order and bonds; dry: a sizing
// pass that allocates no plan buffer (see Plan::dry).
std::unique_ptr<Plan> build_plan(tnx_network* net, const std::string& key, const std::string& order, bool dry) {
  std::unique_ptr<Plan> p(new Plan());
  p->dry = dry;
  static uint64_t serial = 0;
  p->serial = ++serial;
  p->ctx = net->ctx;
  p->prec = net->prec;
  p->narrow_tiles = net->narrow_tiles;
  p->key = key;
  p->order = order;
  p->nin = (int)net->ts.size();
  for (int i = 0; i < p->nin; ++i) {
    const tnx_tensor* t = net->ts[i].t;
    p->new_slot(t->data, t->rank == 0 ? 1 : t->nelem);
  }
  {
    std::vector<BondD> ob;
    for (auto& l : net->tout) {
      for (auto& t : net->ts)
        for (size_t j = 0; j < t.labels.size(); ++j)
          if (t.labels[j] == l) ob.push_back(t.t->bonds[t.perm[j]]);
    }
    std::vector<int32_t> q;
    int64_t nb = 0;
    enumerate_blocks(ob, q, nb);
    int64_t ne = ob.empty() ? 1 : 0;
    for (int64_t b = 0; b < nb && !ob.empty(); ++b) {
      int64_t n = 1;
      for (size_t j = 0; j < ob.size(); ++j) n *= ob[j].deg[q[b * ob.size() + j]];
      ne += n;
    }
    p->out_slot = p->new_slot(nullptr, ne);
  }
  p->d_status = (int32_t*)p->alloc_zero(64);
  if (p->nin > 64) fail(TNX_ERR_UNSUPPORTED, "at most 64 tensors per network");
  std::function<uint64_t(int)> leaves = [&](int node) -> uint64_t {
    const TreeNode& n = net->tree[node];
    return n.leaf >= 0 ? (uint64_t)1 << n.leaf : leaves(n.l) | leaves(n.r);
  };
  std::function<OpView(int)> walk = [&](int node) -> OpView {
    const TreeNode& n = net->tree[node];
    if (n.leaf >= 0) return input_view(net->ts[n.leaf], n.leaf);
    OpView A = walk(n.l);
    OpView B = walk(n.r);
    p->steps.emplace_back();
    StepPlan& s = p->steps.back();
    s.leavesA = leaves(n.l);
    s.leavesB = leaves(n.r);
    s.A = std::move(A);
    s.B = std::move(B);
    build_step(*p, s);
    if (p->prec == TNX_PREC_SPLIT_BF16 || p->prec == TNX_PREC_SPLIT_F16 || p->prec == TNX_PREC_TF32)
      build_split_parts(*p, s);
    return p->steps.back().C;
  };
  OpView root = walk(net->root);
  build_final(*p, root, net->tout);
  fuse_skinny_steps(*p);
  fold_final(*p);
  const char* dbg = dry ? nullptr : getenv("TNX_DEBUG_PLAN");
  if (dbg) {
    if (*dbg && *dbg != '0') {
      auto stats = [](const TaskList& t) {
        int tr = 0, packed = 0, band = 0;
        for (auto& c : t.hchunks) {
          if (c.z == -1) ++tr;
          else if (c.z == -2) ++band;
          else if (c.z > 1) ++packed;
        }
        return std::to_string(t.n) + " tasks, " + std::to_string(t.total) + " elems, " + std::to_string(t.nchunks) +
               " chunks (" + std::to_string(tr) + " transpose tiles, " + std::to_string(band) + " band tiles, " +
               std::to_string(packed) + " packed)";
      };
      fprintf(stderr, "[tnx plan] order %s prec %d\n", p->order.c_str(), p->prec);
      for (size_t i = 0; i < p->steps.size(); ++i) {
        const StepPlan& s = p->steps[i];
        fprintf(stderr, "[tnx plan] step %zu: G=%d flops=%.3e skinny=%.3e tiles=%d skinny_tiles=%d split_tiles=%d\n", i,
                s.G, s.flops, s.flops_skinny, s.ntiles, s.nstiles_skinny, s.nstiles);
        fprintf(stderr, "[tnx plan]   A: %s%s\n[tnx plan]   B: %s%s\n", stats(s.copyA).c_str(),
                s.skipA ? " (done by the fused step)" : "", stats(s.copyB).c_str(),
                s.skipB ? " (done by the fused step)" : "");
        if (s.nftiles)
          fprintf(stderr, "[tnx plan]   fused skinny: %d tiles, output %s\n", s.nftiles,
                  s.fscatter ? "scattered into the next operand" : "written to C");
      }
      fprintf(stderr, "[tnx plan] final: %s\n", stats(p->fin).c_str());
    }
  }
  p->d_slots = (double**)p->alloc_zero(p->h_slots.size() * sizeof(double*));
  p->h_slots_dev.assign(p->h_slots.size(), nullptr);
  CUDA_CHECK(cudaStreamSynchronize(net->ctx->stream));
  return p;
}

Plan* ensure_plan(tnx_network* net) {
  ensure_order(net);
  const std::string order = tree_string(net, net->root);
  const std::string key = plan_key(net, order);
  if (net->plan && net->plan->key == key) return net->plan.get();
  net->plan.reset();
  net->plan = build_plan(net, key, order, false);
  return net->plan.get();
}

void sync_slots(Plan& p, cudaStream_t st) {
  if (p.h_slots == p.h_slots_dev) return;
  CUDA_CHECK(cudaMemcpyAsync(p.d_slots, p.h_slots.data(), p.h_slots.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  p.h_slots_dev = p.h_slots;
}


void enqueue_split(Plan& p, StepPlan& s, cudaStream_t st, bool needA, bool needB, bool balance);

// Enqueue one apply.  `fixed`: network tensors whose data has not changed since
// the previous apply of this plan (a Lanczos solve marks every tensor but the
// vector).  Operands built only from fixed tensors keep their packed and sliced
// forms from that previous apply, and a step whose two operands are both fixed
// keeps its product: neither is recomputed.
// skip_slot >= 0: the relayout of that input tensor was done already (a Lanczos
// step fuses it with its normalisation).
// vary: network tensors that may change between the applies of a sequence
// (a Lanczos solve: the vector).  A split step is K-balanced from its A
// operand unless A varies while B stays fixed (B's slices would then need A's
// exponents of every apply); the choice is the same for every apply of the
// sequence, so slices kept from a previous apply stay consistent.
// skip_slice_step / skip_slice_A: the slices of that step's A (or B) operand
// were written by the caller already (the Lanczos vector mode of the slicing).
void enqueue_plan(Plan& p, cudaStream_t st, uint64_t fixed = 0, int skip_slot = -1, uint64_t vary = ~(uint64_t)0,
                  int skip_slice_step = -1, bool skip_slice_A = true) {
  tnx_ctx* c = p.ctx;
  for (size_t si = 0; si < p.steps.size(); ++si) {
    StepPlan& s = p.steps[si];
    const bool needA = (s.leavesA & ~fixed) != 0;
    const bool needB = (s.leavesB & ~fixed) != 0;
    if (!needA && !needB) continue;
    // relayouts of A and B, unless a fused step (or the caller) does them
    const bool copyA = needA && !s.skipA && !s.nftiles && (skip_slot < 0 || s.A.slot != skip_slot);
    const bool copyB = needB && !s.skipB && (skip_slot < 0 || s.B.slot != skip_slot);
    if (copyA || copyB) {
      ProfScope ps(c, st, TNX_KC_RELAYOUT,
                   16.0 * (double)((copyA ? s.copyA.total : 0) + (copyB ? s.copyB.total : 0)));
      if (copyA) CUDA_CHECK(tnx_launch_copy(s.copyA.d, s.copyA.chunks, s.copyA.nchunks, p.d_slots, st));
      if (copyB) CUDA_CHECK(tnx_launch_copy(s.copyB.d, s.copyB.chunks, s.copyB.nchunks, p.d_slots, st));
    }
    if (s.nftiles) {
      ProfScope ps(c, st, TNX_KC_SKINNY, s.flops_skinny);
      CUDA_CHECK(tnx_launch_fused_skinny(s.dG, s.dFT, s.nftiles, s.dFC, s.fkp, s.fnp, p.d_slots, st));
    } else if (s.nstiles_skinny) {
      ProfScope ps(c, st, TNX_KC_SKINNY, s.flops_skinny);
      CUDA_CHECK(tnx_launch_gemm_skinny(s.dG, s.dTs, s.nstiles_skinny, p.d_slots, st));
    }
    switch (p.prec) {
      case TNX_PREC_F64: {
        ProfScope ps(c, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
        CUDA_CHECK(tnx_launch_gemm_f64(s.dG, s.dT, s.ntiles, p.d_slots, st));
        break;
      }
      case TNX_PREC_F32: {
        ProfScope ps(c, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
        CUDA_CHECK(tnx_launch_gemm_f32(s.dG, s.dT, s.ntiles, p.d_slots, st));
        break;
      }
      default: {
        const bool balance = !((s.leavesA & vary) != 0 && (s.leavesB & vary) == 0);
        const bool pre = (int)si == skip_slice_step;
        enqueue_split(p, s, st, needA && !(pre && skip_slice_A), needB && !(pre && !skip_slice_A), balance);
        break;
      }
    }
  }
  if (p.fin_folded) return;   // the last product's epilogue wrote the output
  ProfScope ps(c, st, TNX_KC_FINAL, 16.0 * (double)p.fin.total);
  CUDA_CHECK(tnx_launch_copy(p.fin.d, p.fin.chunks, p.fin.nchunks, p.d_slots, st));
}

// Stream capture of `body` into g (graphs need a non-default stream).
void capture_graph(tnx_ctx* c, cudaStream_t st, GraphRec& g, const std::function<void()>& body) {
  g.prof = c->prof;
  c->capture_recs = &g.recs;
  g.nlaunch = 0;
  tnx_count_into(&g.nlaunch);
  CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  try {
    body();
  } catch (...) {
    tnx_count_into(nullptr);
    cudaGraph_t gr = nullptr;
    cudaStreamEndCapture(st, &gr);
    if (gr) cudaGraphDestroy(gr);
    c->capture_recs = nullptr;
    throw;
  }
  tnx_count_into(nullptr);
  c->capture_recs = nullptr;
  cudaGraph_t gr = nullptr;
  CUDA_CHECK(cudaStreamEndCapture(st, &gr));
  cudaError_t e = cudaGraphInstantiate(&g.exec, gr, 0);
  cudaGraphDestroy(gr);
  CUDA_CHECK(e);
}


void bind_inputs(tnx_network* net, Plan& p) {
  for (int i = 0; i < p.nin; ++i) p.h_slots[i] = net->ts[i].t->data;
}

void check_out_bonds(const Plan& p, const tnx_tensor* out) {
  if ((int)p.out_bonds.size() != out->rank) fail(TNX_ERR_BOND_MISMATCH, "output rank differs from TOUT");
  for (int j = 0; j < out->rank; ++j)
    if (out->bonds[j] != p.out_bonds[j]) fail(TNX_ERR_BOND_MISMATCH, "output bonds differ from the TOUT bonds");
}

}  // namespace

namespace {
void build_split_parts(Plan& p, StepPlan& s) { tnx_build_split_parts(p, s); }
void enqueue_split(Plan& p, StepPlan& s, cudaStream_t st, bool needA, bool needB, bool balance) {
  tnx_enqueue_split(p, s, st, needA, needB, balance);
}
}  // namespace

// shared with the batch and serving modules
Plan* tnx_ensure_plan(tnx_network* net) { return ensure_plan(net); }

// One apply of the network into `out`, enqueued on `st` (a CUDA graph when
// graphs are on and st is not the legacy default stream).
void tnx_apply_enqueue(tnx_network* net, tnx_tensor* out, cudaStream_t st) {
  Plan* p = ensure_plan(net);
  check_out_bonds(*p, out);
  bind_inputs(net, *p);
  p->h_slots[p->out_slot] = out->data;
  sync_slots(*p, st);
  tnx_ctx* c = net->ctx;
  // The first apply of a plan runs eagerly; the graph is captured from the
  // second on (a plan applied once, as in a DMRG sweep where every bond brings
  // new bond dimensions, would pay capture and instantiation for one replay).
  if (st != nullptr && c->use_graphs && !p->apply_graph && p->eager_applies == 0) {
    ++p->eager_applies;
    enqueue_plan(*p, st);
  } else if (st != nullptr && c->use_graphs) {
    if (!p->apply_graph || p->apply_graph->prof != c->prof) {
      p->apply_graph.reset(new GraphRec());
      capture_graph(c, st, *p->apply_graph, [&] { enqueue_plan(*p, st); });
    }
    CUDA_CHECK(cudaGraphLaunch(p->apply_graph->exec, st));
    tnx_note_launch(p->apply_graph->nlaunch);
    if (c->prof) {
      CUDA_CHECK(cudaStreamSynchronize(st));
      prof_accumulate(c, p->apply_graph->recs);
    }
  } else {
    enqueue_plan(*p, st);
  }
}
void tnx_bind_inputs(tnx_network* net, Plan& p) { bind_inputs(net, p); }
void tnx_check_out_bonds(const Plan& p, const tnx_tensor* out) { check_out_bonds(p, out); }
void tnx_capture_graph(tnx_ctx* c, cudaStream_t st, GraphRec& g, const std::function<void()>& body) {
  capture_graph(c, st, g, body);
}

// ------------------------------------------------------------------ C-ABI
static bool all_put(const tnx_network* net);

extern "C" tnx_status tnx_network_create(tnx_ctx* ctx, const char* spec, tnx_network** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || !spec || !out) fail(TNX_ERR_ARG, "null argument");
    std::unique_ptr<tnx_network> net(new tnx_network());
    net->ctx = ctx;
    std::string text(spec), line, order;
    bool have_tout = false;
    size_t p0 = 0;
    while (p0 <= text.size()) {
      size_t p1 = text.find('\n', p0);
      if (p1 == std::string::npos) p1 = text.size();
      line = trim(text.substr(p0, p1 - p0));
      p0 = p1 + 1;
      if (line.empty() || line[0] == '#') continue;   // comment lines (Sec. 8.4 network file)
      size_t c = line.find(':');
      if (c == std::string::npos) fail(TNX_ERR_NETWORK, "line without ':' : " + line);
      std::string key = trim(line.substr(0, c)), rest = trim(line.substr(c + 1));
      if (key == "TOUT") {
        net->tout = split_labels(rest);
        have_tout = true;
      } else if (key == "ORDER") {
        order = rest;
      } else {
        if (!valid_name(key)) fail(TNX_ERR_NETWORK, "bad tensor name '" + key + "'");
        for (auto& t : net->ts)
          if (t.name == key) fail(TNX_ERR_NETWORK, "duplicate tensor name '" + key + "'");
        NetTensor nt;
        nt.name = key;
        nt.labels = split_labels(rest);
        std::set<std::string> u(nt.labels.begin(), nt.labels.end());
        if (u.size() != nt.labels.size()) fail(TNX_ERR_NETWORK, "a label appears twice on tensor '" + key + "'");
        if ((int)nt.labels.size() > TNX_MAXR) fail(TNX_ERR_UNSUPPORTED, "tensor rank above the limit");
        net->ts.push_back(nt);
      }
    }
    if (!have_tout) fail(TNX_ERR_NETWORK, "missing TOUT");
    if (net->ts.empty()) fail(TNX_ERR_NETWORK, "no tensors");
    std::map<std::string, int> cnt;
    for (auto& t : net->ts)
      for (auto& l : t.labels) cnt[l]++;
    std::set<std::string> open;
    for (auto& kv : cnt) {
      if (kv.second > 2) fail(TNX_ERR_NETWORK, "label '" + kv.first + "' appears on more than two tensors");
      if (kv.second == 1) open.insert(kv.first);
    }
    std::set<std::string> to(net->tout.begin(), net->tout.end());
    if (to.size() != net->tout.size() || to != open) fail(TNX_ERR_NETWORK, "TOUT must list exactly the open labels");
    if (!order.empty()) set_tree_from_string(net.get(), order);
    else set_default_tree(net.get());
    *out = net.release();
  });
}

extern "C" tnx_status tnx_network_destroy(tnx_network* net) {
  if (!net) return TNX_ERR_ARG;
  cudaStreamSynchronize(net->ctx->stream);
  delete net;
  return TNX_OK;
}

extern "C" tnx_status tnx_network_put(tnx_network* net, const char* name, tnx_tensor* t, int nlab,
                                      const char* const* labels) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    if (!name || !t) fail(TNX_ERR_ARG, "null argument");
    NetTensor* nt = nullptr;
    for (auto& x : net->ts)
      if (x.name == name) nt = &x;
    if (!nt) fail(TNX_ERR_NETWORK, std::string("no tensor named '") + name + "' in the network");
    const int r = (int)nt->labels.size();
    if (t->rank != r) fail(TNX_ERR_NETWORK, "rank of the tensor differs from the blueprint");
    std::vector<int> perm(r);
    if (!labels) {
      std::iota(perm.begin(), perm.end(), 0);
    } else {
      if (nlab != r) fail(TNX_ERR_NETWORK, "one label per leg is required");
      std::vector<int> used(r, 0);
      for (int j = 0; j < r; ++j) {
        int found = -1;
        for (int i = 0; i < r; ++i)
          if (labels[i] && nt->labels[j] == labels[i]) found = i;
        if (found < 0 || used[found]) fail(TNX_ERR_NETWORK, "labels must be a permutation of the blueprint labels");
        used[found] = 1;
        perm[j] = found;
      }
    }
    nt->t = t;
    nt->perm = perm;
  });
}

extern "C" tnx_status tnx_network_set_order(tnx_network* net, int optimal, const char* order) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    if (optimal) {
      if (optimal != 1 && optimal != 2) fail(TNX_ERR_ARG, "optimal must be 0, 1 or 2");
      net->optimal = optimal;
      net->order_dims_key.clear();
      if (all_put(net)) ensure_order(net);
    } else {
      if (!order || !*order) fail(TNX_ERR_NETWORK, "an explicit order is required when optimal is off");
      set_tree_from_string(net, order);
      net->optimal = 0;
    }
  });
}

static bool all_put(const tnx_network* net) {
  for (auto& t : net->ts)
    if (!t.t) return false;
  return true;
}

// With optimal on and every tensor loaded, the tree reflects the loaded
// dimensions (computed now, or reused while the dimensions are unchanged).
extern "C" tnx_status tnx_network_get_order(const tnx_network* cnet, char* buf, size_t len) {
  if (!cnet || !buf) return TNX_ERR_ARG;
  tnx_network* net = const_cast<tnx_network*>(cnet);
  return tnx_guard(net->ctx, [&] {
    if (net->optimal && all_put(net)) ensure_order(net);
    std::string s = tree_string(net, net->root);
    if (s.size() + 1 > len) fail(TNX_ERR_ARG, "buffer too small for the order string");
    memcpy(buf, s.c_str(), s.size() + 1);
  });
}

extern "C" tnx_status tnx_network_set_precision(tnx_network* net, int prec) {
  if (!net) return TNX_ERR_ARG;
  if (prec < TNX_PREC_F64 || prec > TNX_PREC_TF32) return TNX_ERR_ARG;
  net->prec = prec;
  return TNX_OK;
}

extern "C" tnx_status tnx_network_launch_into(tnx_network* net, tnx_tensor* out) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    if (!out) fail(TNX_ERR_ARG, "null output");
    tnx_apply_enqueue(net, out, net->ctx->stream);
  });
}

extern "C" tnx_status tnx_network_launch(tnx_network* net, tnx_tensor** out) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    if (!out) fail(TNX_ERR_ARG, "null output");
    Plan* p = ensure_plan(net);
    std::unique_ptr<tnx_tensor> t(make_tensor(net->ctx, p->out_bonds));
    tnx_status s = tnx_network_launch_into(net, t.get());
    if (s != TNX_OK) throw TnxError{s, net->ctx->err};
    *out = t.release();
  });
}

extern "C" tnx_status tnx_network_flops(tnx_network* net, double* flops) {
  if (!net || !flops) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    Plan* p = ensure_plan(net);
    double f = 0;
    for (auto& s : p->steps) f += s.flops;
    *flops = f;
  });
}

extern "C" tnx_status tnx_network_nsteps(tnx_network* net, int* nsteps) {
  if (!net || !nsteps) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] { *nsteps = (int)ensure_plan(net)->steps.size(); });
}

extern "C" tnx_status tnx_network_step_sizes(tnx_network* net, int step, int* ngroups, int* nsym, int64_t* nA,
                                             int64_t* nB) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    Plan* p = ensure_plan(net);
    if (step < 0 || step >= (int)p->steps.size()) fail(TNX_ERR_ARG, "step out of range");
    const StepPlan& s = p->steps[step];
    if (ngroups) *ngroups = s.G;
    if (nsym) *nsym = s.nsym;
    if (nA) *nA = s.A.nblk;
    if (nB) *nB = s.B.nblk;
  });
}

extern "C" tnx_status tnx_network_step_tables(tnx_network* net, int step, int32_t* charges, int64_t* mkn,
                                              int64_t* amap, int64_t* bmap) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    Plan* p = ensure_plan(net);
    if (step < 0 || step >= (int)p->steps.size()) fail(TNX_ERR_ARG, "step out of range");
    const StepPlan& s = p->steps[step];
    if (charges) std::copy(s.charges.begin(), s.charges.end(), charges);
    if (mkn) std::copy(s.mkn.begin(), s.mkn.end(), mkn);
    if (amap) std::copy(s.amap.begin(), s.amap.end(), amap);
    if (bmap) std::copy(s.bmap.begin(), s.bmap.end(), bmap);
  });
}

// ---------------------------------------------------------------- Lanczos
// Workspace and captured graph of a Lanczos solve, reused while the plan, the
// step count and the bound buffers stay the same.
struct LanczosCache {
  uint64_t plan_serial = 0;
  int nsteps = 0, slot = -1;
  int64_t n = 0;
  const double* v0 = nullptr;
  double* evec = nullptr;
  std::vector<std::unique_ptr<DevBuf>> bufs;
  LanczosDev L;
  std::unique_ptr<GraphRec> graph;
  int eager_runs = 0;
  // vector mode of the slicing (see vector_slicing_tables): decided once per cache
  bool vs_decided = false;
  int vs_step = -1;                // the step whose operand is sliced straight from w (-1: not used)
  bool vs_sideA = true;
  std::unique_ptr<DevBuf> vs_rowtab, vs_jobs;
  const int2* vs_items = nullptr;
  int64_t vs_nitems = 0;
};

tnx_network::~tnx_network() = default;

namespace {
// Bytes of the Lanczos workspace buffers, in allocation order: V, w, alpha,
// beta, coef, partial sums, y, scratch, state, eval, omega.
std::vector<size_t> lanczos_buffer_sizes(int64_t n, int nsteps) {
  return {(size_t)(nsteps + 1) * n * 8, (size_t)n * 8, (size_t)(nsteps + 1) * 8, (size_t)(nsteps + 2) * 8,
          (size_t)(nsteps + 2) * 8, (size_t)std::max<int64_t>(1216, (int64_t)608 * (nsteps + 2)) * 8,
          (size_t)(nsteps + 1) * 8, (size_t)(4 * (nsteps + 1)) * 8, 64, 64, (size_t)(2 * (nsteps + 2)) * 8};
}
}  // namespace

size_t tnx_lanczos_workspace_bytes(int64_t n, int nsteps) {
  size_t b = 0;
  for (size_t x : lanczos_buffer_sizes(n, nsteps)) b += std::max<size_t>(x, 256);
  return b;
}

// The Lanczos vector mode of the slicing: when the only reader of the vector is
// a plain relayout into a split product's operand that is sliced without K
// balancing, and every packed row of that operand takes its K entries from one
// contiguous run of the vector, the next apply's slices of the operand are
// written straight from w at the end of a step, together with v_{j+1} = w /
// beta_{j+1}: the FP64 packed operand is never formed.  rowtab[base(job) + row]
// = offset in the vector of that packed row's K entries; jobs are the step's
// slicing jobs with src_off = base(job).  Every element of every task is
// mapped (the tasks may have merged or dropped legs in any order); false, with
// nothing built, when a row's entries are not one run in order or a row is not
// filled exactly once.
bool vector_slicing_tables(const TaskList& vc, const std::vector<SliceJob>& jobs, std::vector<int64_t>& rowtab,
                           std::vector<SliceJob>& vjobs) {
  if (jobs.empty() || vc.h.empty()) return false;
  std::vector<int64_t> base(jobs.size() + 1, 0);
  for (size_t b = 0; b < jobs.size(); ++b) {
    if (jobs[b].rows < 0 || jobs[b].ld < jobs[b].K || jobs[b].K < 1) return false;
    base[b + 1] = base[b] + jobs[b].rows;
  }
  rowtab.assign((size_t)base.back(), -1);
  std::vector<int32_t> cnt((size_t)base.back(), 0);
  // jobs by their start in the operand slot
  std::vector<int> ord(jobs.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return jobs[a].src_off < jobs[b].src_off; });
  auto find_job = [&](int64_t P) {
    int lo = 0, hi = (int)ord.size() - 1, f = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) / 2;
      if (jobs[ord[mid]].src_off <= P) {
        f = ord[mid];
        lo = mid + 1;
      } else {
        hi = mid - 1;
      }
    }
    return f;
  };
  int f = -1;   // the job of the previous element (consecutive elements mostly share it)
  for (const CopyTask& t : vc.h) {
    const int r = t.rank;
    if (t.tleg != -1 || r < 1 || r > TNX_MAXR) return false;
    int64_t idx[TNX_MAXR] = {0};
    int64_t so = 0, dof = 0;
    for (int64_t e = 0; e < t.nelem; ++e) {
      const int64_t P = t.dst_off + dof;
      if (f < 0 || P < jobs[f].src_off || P >= jobs[f].src_off + (int64_t)jobs[f].rows * jobs[f].ld) f = find_job(P);
      if (f < 0) return false;
      const SliceJob& jb = jobs[f];
      if (jb.src_slot != t.dst_slot) return false;
      const int64_t off = P - jb.src_off, row = off / jb.ld, k = off % jb.ld;
      if (row >= jb.rows || k >= jb.K) return false;
      const size_t ri = (size_t)(base[f] + row);
      const int64_t start = t.src_off + so - k;   // where entry 0 of this row must lie
      if (rowtab[ri] == -1) rowtab[ri] = start;
      else if (rowtab[ri] != start) return false;
      ++cnt[ri];
      // next element: the last leg fastest
      for (int l = r - 1; l >= 0; --l) {
        so += t.sstride[l];
        dof += t.dstride[l];
        if (++idx[l] < t.shape[l]) break;
        so -= (int64_t)t.shape[l] * t.sstride[l];
        dof -= (int64_t)t.shape[l] * t.dstride[l];
        idx[l] = 0;
      }
    }
  }
  for (size_t b = 0; b < jobs.size(); ++b)
    for (int64_t row = 0; row < jobs[b].rows; ++row) {
      const size_t ri = (size_t)(base[b] + row);
      if (rowtab[ri] < 0 || cnt[ri] != jobs[b].K) return false;   // a row not filled exactly once
    }
  vjobs = jobs;
  for (size_t b = 0; b < jobs.size(); ++b) vjobs[b].src_off = base[b];
  return true;
}

// A whole Lanczos solve enqueued on `st`; at its end the eigenvalue and the
// number of matvecs are copied to host_out[0] (double) and host_out[1] (int32
// in its first four bytes), which must be pinned host memory.  No sync.
void tnx_lanczos_enqueue(tnx_network* net, int slot, tnx_tensor* v0, int nsteps, tnx_tensor* evec, cudaStream_t st,
                         double* host_out) {
  tnx_ctx* ctx = net->ctx;
  NetTensor& vt = net->ts[slot];
  if (!vt.t) {
    vt.t = v0;
    vt.perm.assign(v0->rank, 0);
    std::iota(vt.perm.begin(), vt.perm.end(), 0);
  }
  for (int j = 0; j < (int)vt.perm.size(); ++j)
    if (vt.perm[j] != j) fail(TNX_ERR_NETWORK, "the vector slot must be put in blueprint leg order");
  if (v0->bonds != vt.t->bonds) fail(TNX_ERR_BOND_MISMATCH, "v0 bonds differ from the vector slot's bonds");
  Plan* p = ensure_plan(net);
  if (p->out_bonds != v0->bonds) fail(TNX_ERR_BOND_MISMATCH, "the operator's output bonds differ from the vector's");
  if (evec) check_out_bonds(*p, evec);
  const int64_t n = v0->nelem;
  std::unique_ptr<LanczosCache>& lc = net->lanczos;
  if (!lc || lc->plan_serial != p->serial || lc->nsteps != nsteps || lc->n != n || lc->slot != slot) {
    lc.reset(new LanczosCache());
    lc->plan_serial = p->serial;
    lc->nsteps = nsteps;
    lc->n = n;
    lc->slot = slot;
    LanczosDev& L = lc->L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.nmax = nsteps;
    L.nblocks = tnx_reduce_blocks(n);
    const std::vector<size_t> sz = lanczos_buffer_sizes(n, nsteps);
    size_t next = 0;
    auto dev = [&](size_t bytes) {
      if (bytes != sz[next++]) fail(TNX_ERR_ARG, "internal: Lanczos workspace sizes disagree");
      lc->bufs.emplace_back(new DevBuf(ctx, std::max<size_t>(bytes, 256)));
      CUDA_CHECK(cudaMemsetAsync(lc->bufs.back()->p, 0, std::max<size_t>(bytes, 256), st));
      return lc->bufs.back()->p;
    };
    L.V = (double*)dev(sz[0]);
    L.w = (double*)dev(sz[1]);
    L.alpha = (double*)dev(sz[2]);
    L.beta = (double*)dev(sz[3]);
    L.coef = (double*)dev(sz[4]);
    L.partial = (double*)dev(sz[5]);
    L.y = (double*)dev(sz[6]);
    L.scratch = (double*)dev(sz[7]);
    L.state = (int32_t*)dev(sz[8]);
    L.eval = (double*)dev(sz[9]);
    L.omega = (double*)dev(sz[10]);
  }
  LanczosDev& L = lc->L;
  bind_inputs(net, *p);
  p->h_slots[p->out_slot] = L.w;
  sync_slots(*p, st);
  double* evp = evec ? evec->data : nullptr;
  // apply 0 prepares every operand; later applies only those fed by the vector
  const uint64_t fixed = ~((uint64_t)1 << slot);
  // When exactly one relayout reads the vector (plain tasks only, no fused
  // step gathering it), v_{j+1} = w / beta_{j+1} and that relayout of v_{j+1}
  // are one launch at the end of step j, and apply j+1 skips the relayout.
  const TaskList* vcopy = nullptr;
  {
    int readers = 0;
    for (auto& s : p->steps) {
      if (s.A.slot == slot) {
        ++readers;
        vcopy = s.nftiles ? nullptr : &s.copyA;
      }
      if (s.B.slot == slot) {
        ++readers;
        vcopy = &s.copyB;
      }
    }
    if (readers != 1) vcopy = nullptr;
    if (vcopy)
      for (const CopyTask& t : vcopy->h)
        if (t.tleg < -1 || t.src_slot != slot) vcopy = nullptr;
  }
  // the relayout reads every entry of the vector once (each block of the vector
  // is one task): it also writes v_{j+1} itself
  int vfull = 0;
  if (vcopy) {
    int64_t cover = 0;
    std::set<int64_t> starts;
    for (const CopyTask& t : vcopy->h) {
      cover += t.nelem;
      starts.insert(t.src_off);
    }
    vfull = cover == n && starts.size() == vcopy->h.size() && vcopy->h.size() == (size_t)v0->nblk ? 1 : 0;
  }
  // vector mode of the slicing (split precisions only, and only for an operand
  // the Lanczos applies slice without K balancing)
  if (!lc->vs_decided) {
    lc->vs_decided = true;
    const bool split = p->prec == TNX_PREC_SPLIT_BF16 || p->prec == TNX_PREC_SPLIT_F16;
    if (split && vcopy && vfull) {
      for (size_t si = 0; si < p->steps.size(); ++si) {
        StepPlan& s = p->steps[si];
        const bool sideA = vcopy == &s.copyA, sideB = vcopy == &s.copyB;
        if (!sideA && !sideB) continue;
        const uint64_t vary = ~fixed;
        const bool balance = !((s.leavesA & vary) != 0 && (s.leavesB & vary) == 0);
        const bool other = sideA ? (s.leavesB & ~fixed) != 0 : (s.leavesA & ~fixed) != 0;
        const StepPlan::Jobs& J = sideA ? s.jobsA : s.jobsB;
        std::vector<int64_t> rowtab;
        std::vector<SliceJob> vjobs;
        if (!balance && !other && !s.nftiles && J.n > 0 && J.nitems > 0 &&
            vector_slicing_tables(*vcopy, J.h, rowtab, vjobs)) {
          lc->vs_rowtab.reset(new DevBuf(ctx, std::max<size_t>(rowtab.size() * 8, 256)));
          lc->vs_jobs.reset(new DevBuf(ctx, std::max<size_t>(vjobs.size() * sizeof(SliceJob), 256)));
          CUDA_CHECK(cudaMemcpyAsync(lc->vs_rowtab->p, rowtab.data(), rowtab.size() * 8, cudaMemcpyHostToDevice, st));
          CUDA_CHECK(cudaMemcpyAsync(lc->vs_jobs->p, vjobs.data(), vjobs.size() * sizeof(SliceJob),
                                     cudaMemcpyHostToDevice, st));
          CUDA_CHECK(cudaStreamSynchronize(st));   // the host tables are freed on return
          lc->vs_step = (int)si;
          lc->vs_sideA = sideA;
          lc->vs_items = J.items;
          lc->vs_nitems = J.nitems;
        }
        break;
      }
    }
  }
  const bool vslice = lc->vs_step >= 0;
  auto body = [&] {
    {
      ProfScope ps(ctx, st, TNX_KC_VECTOR, 24.0 * (double)n);
      CUDA_CHECK(tnx_launch_lanczos_init(L, v0->data, st));
    }
    for (int j = 0; j < nsteps; ++j) {
      // the input slot points at v_0 here; each step kernel points it at v_{j+1}
      if (j == 0) CUDA_CHECK(tnx_launch_lanczos_set_input(p->d_slots + slot, L, 0, st));
      {
        // TNX_PROF_LAST_APPLY: the events of the earlier applies are left out
        const uint32_t prof = ctx->prof;
        if ((prof & TNX_PROF_LAST_APPLY) && j != nsteps - 1) ctx->prof = 0;
        try {
          enqueue_plan(*p, st, j == 0 ? 0 : fixed, (j > 0 && vcopy) ? slot : -1, ~fixed,
                       (j > 0 && vslice) ? lc->vs_step : -1, lc->vs_sideA);
        } catch (...) {
          ctx->prof = prof;
          throw;
        }
        ctx->prof = prof;
      }
      // bytes of a step without the Gram-Schmidt pass: alpha (2n), the
      // three-term step with the norm (4n), scale (2n); a step that takes the
      // pass (decided on the device) adds (j+1)n + n for the dots and
      // (j+1)n + 2n for the update
      ProfScope ps(ctx, st, TNX_KC_VECTOR, 8.0 * (double)n * 8);
      CUDA_CHECK(tnx_launch_lanczos_step(L, j, p->d_slots + slot, st, vcopy == nullptr,
                                         p->prec == TNX_PREC_F32 || p->prec == TNX_PREC_TF32));
      if (vslice) {
        // v_{j+1} and the next apply's slices of the vector operand in one pass over w
        const VecSrc vs{(const int64_t*)lc->vs_rowtab->p, L.w, L.V + (int64_t)(j + 1) * n,
                        L.scratch + 3 * L.nmax + 3, L.state};
        CUDA_CHECK(tnx_launch_slices_vec((const SliceJob*)lc->vs_jobs->p, lc->vs_items, lc->vs_nitems, p->nslice,
                                         p->beta, p->prec == TNX_PREC_SPLIT_F16 ? 1 : 0, p->d_slots, vs, st));
      } else if (vcopy) {
        CUDA_CHECK(tnx_launch_copy_scaled(vcopy->d, vcopy->chunks, vcopy->nchunks, p->d_slots, L.w,
                                          L.V + (int64_t)(j + 1) * n, n, vfull, L.scratch + 3 * L.nmax + 3, L.state,
                                          st));
      }
    }
    ProfScope ps(ctx, st, TNX_KC_VECTOR, evp ? 8.0 * (double)n * (nsteps + 2) : 0.0);
    CUDA_CHECK(tnx_launch_lanczos_finish(L, evp, st));
  };
  if (st != nullptr && ctx->use_graphs && !lc->graph && lc->eager_runs == 0) {
    ++lc->eager_runs;   // the first solve of a plan runs eagerly (see tnx_apply_enqueue)
    body();
  } else if (st != nullptr && ctx->use_graphs) {
    if (!lc->graph || lc->v0 != v0->data || lc->evec != evp || lc->graph->prof != ctx->prof) {
      lc->graph.reset(new GraphRec());
      lc->v0 = v0->data;
      lc->evec = evp;
      capture_graph(ctx, st, *lc->graph, body);
    }
    CUDA_CHECK(cudaGraphLaunch(lc->graph->exec, st));
    tnx_note_launch(lc->graph->nlaunch);
  } else {
    body();
  }
  // the device slot of the vector now points into L.V: restore the table next time
  p->h_slots_dev.assign(p->h_slots.size(), nullptr);
  CUDA_CHECK(cudaMemcpyAsync(host_out, L.eval, 8, cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaMemcpyAsync(host_out + 1, L.state, 8, cudaMemcpyDeviceToHost, st));
}

size_t tnx_network_plan_bytes(tnx_network* net) {
  ensure_order(net);
  const std::string order = tree_string(net, net->root);
  const std::string key = plan_key(net, order);
  if (net->plan && net->plan->key == key) {
    size_t b = 0;
    for (auto& d : net->plan->bufs) b += d->bytes;
    return b;
  }
  if (net->sized_key != key) {
    std::unique_ptr<Plan> p = build_plan(net, key, order, true);
    net->sized_key = key;
    net->sized_bytes = p->dry_bytes;
  }
  return net->sized_bytes;
}

size_t tnx_network_lanczos_bytes(tnx_network* net) {
  size_t b = 0;
  if (net->lanczos)
    for (auto& d : net->lanczos->bufs) b += d->bytes;
  return b;
}

// Device bytes held by the network's plan and Lanczos workspace.
size_t tnx_network_resident_bytes(tnx_network* net) {
  size_t b = 0;
  if (net->plan)
    for (auto& d : net->plan->bufs) b += d->bytes;
  if (net->lanczos)
    for (auto& d : net->lanczos->bufs) b += d->bytes;
  return b;
}

// Frees the plan and the Lanczos workspace (rebuilt on the next use).  The
// caller guarantees nothing of this network is in flight.
void tnx_network_evict(tnx_network* net) {
  net->lanczos.reset();
  net->plan.reset();
}

int tnx_network_slot(tnx_network* net, const char* name) {
  for (size_t i = 0; i < net->ts.size(); ++i)
    if (net->ts[i].name == name) return (int)i;
  return -1;
}

extern "C" tnx_status tnx_network_resident(tnx_network* net, size_t* bytes, size_t* plan_bytes) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    if (bytes) *bytes = tnx_network_resident_bytes(net);
    if (plan_bytes) {
      if (!all_put(net)) fail(TNX_ERR_NETWORK, "every tensor must be put before the plan can be sized");
      *plan_bytes = tnx_network_plan_bytes(net);
    }
  });
}

extern "C" tnx_status tnx_lanczos(tnx_network* net, const char* vec_slot, tnx_tensor* v0, int nsteps, double* eval,
                                  tnx_tensor* evec, int* nmatvec) {
  if (!net) return TNX_ERR_ARG;
  return tnx_guard(net->ctx, [&] {
    tnx_ctx* ctx = net->ctx;
    if (!vec_slot || !v0 || !eval || nsteps < 1 || nsteps > 500) fail(TNX_ERR_ARG, "bad Lanczos arguments");
    const int slot = tnx_network_slot(net, vec_slot);
    if (slot < 0) fail(TNX_ERR_NETWORK, std::string("no tensor named '") + vec_slot + "'");
    double* hp = (double*)ctx->pinned;
    tnx_lanczos_enqueue(net, slot, v0, nsteps, evec, ctx->stream, hp);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    // a solve that ran from its graph keeps its profile records there (an eager
    // one, the first of a plan, left them pending on the context)
    if (ctx->stream && ctx->use_graphs && ctx->prof && net->lanczos && net->lanczos->graph)
      prof_accumulate(ctx, net->lanczos->graph->recs);
    check_device_status(ctx);
    *eval = hp[0];
    if (nmatvec) *nmatvec = ((int32_t*)(hp + 1))[0];
  });
}
