/*
 * louvain_oracle.cpp -- TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded CPU statement
 * of the Louvain method as GVE-Louvain (arXiv 2312.04876) describes it, used to check the GPU
 * library.  Only tests/, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It shares no code with the GPU library.
 *
 * What it follows (paper sections / equations / algorithms):
 *   modularity ............ Eq. 1, second form  Q = sum_c [ sigma_c/2m - (Sigma_c/2m)^2 ]
 *   move score ............ Eq. 2 scaled by 2m^2:  N = 2m (K_i->c - K_i->d) - K_i (Sigma_c - Sigma_d + K_i),
 *                           Delta Q = 2N / (2m)^2
 *   pass loop ............. Algorithm 1 (init, local move, convergence tests, renumber, dendrogram
 *                           lookup, aggregation, threshold scaling)
 *   local-moving phase .... Algorithm 2 (pruning flags, best neighbouring community, Sigma update,
 *                           re-mark neighbours, per-iteration tolerance test)
 *   aggregation phase ..... Algorithm 3 (community-vertex CSR by counting, super-vertex rows by
 *                           summing arc weights per neighbouring community, self-loops kept)
 *   dynamic graphs ........ a batch of edge deletions and insertions applied to the CSR, and a run
 *                           whose first pass starts from a given membership (Section 4.2 keeps the
 *                           first pass's graph in a format open to batch updates; Figure 2 feeds
 *                           each later pass an initial membership; the Conclusion names updating
 *                           the memberships of dynamic graphs as the next step)
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   R1  a self-loop is stored once and counts once in K_i, sigma_c and 2m;
 *   R2  candidates = communities of neighbours j != i, the current community d excluded; best = max N,
 *       ties to the smallest community id; move iff N > 0;
 *   R3  deterministic schedule: colour classes of the greedy colouring in decreasing priority
 *       (prio(v) = hash3(seed, pass, v), ties by id); per class all flagged vertices decide against
 *       the class-start state, then all moves apply; marks set by a class make later classes of the
 *       same iteration eligible;
 *   R4  l_i counts executed iterations (1-based, including the one that passes the tolerance test);
 *       the test is (double)(2 sum N) <= tau * ((double)2m)^2 in integer mode;
 *   R5  |Gamma_old| = |V'| of the pass; stop when |Gamma| / |V'| > tau_agg;
 *   R6  renumbering = rank of the id among occupied ids; the final lookup applies only the
 *       membership of a pass that was not aggregated; the output is renumbered the same way;
 *   R7  a moved vertex marks its neighbours j != i.
 * Integer weights use exact int64 (sum N in __int128) and require 2m < 2^31; fp32 weights are
 * widened to double and every sum is double (the paper computes in fp64).
 */
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

typedef __int128 i128;

uint64_t mix64(uint64_t z) {  // SplitMix64 output function (Steele, Lea, Flood 2014)
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
const uint64_t kGamma = 0x9e3779b97f4a7c15ULL;
uint64_t hash3(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t x = mix64(a + kGamma);
  x = mix64(x + b + 2 * kGamma);
  return mix64(x + c + 3 * kGamma);
}

struct Params {
  int32_t max_passes, max_iterations;
  double tolerance, tolerance_drop, aggregation_tolerance;
  int32_t pruning, schedule;  // schedule 0 = colour-synchronous, 1 = sequential asynchronous
  uint64_t seed;
};

struct PassStats {
  int32_t pass, iterations;
  int64_t moves, n_vertices, n_arcs, n_communities;
  double modularity;
};

template <class W>
struct Graph {
  int64_t n = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> tg;
  std::vector<W> w;
};

struct IntArith {
  typedef int64_t W;
  typedef i128 S;
  static const bool is_int = true;
  static bool converged(S sum_n, W two_m, double tau) {
    double lhs = (double)(sum_n * 2);
    double t = (double)two_m;
    return lhs <= tau * (t * t);
  }
  static double modularity(W two_m, W sigma_in, const std::vector<W>& tot) {
    // Q = (2m sum sigma_c - sum Sigma_c^2) / (2m)^2, exact integers, one rounding per operand
    int64_t sq = 0;
    for (W t : tot) sq += t * t;
    int64_t num = two_m * sigma_in - sq, den = two_m * two_m;
    return (double)num / (double)den;
  }
};

struct FpArith {
  typedef double W;
  typedef double S;
  static const bool is_int = false;
  static bool converged(S sum_n, W two_m, double tau) { return 2.0 * sum_n <= tau * (two_m * two_m); }
  static double modularity(W two_m, W sigma_in, const std::vector<W>& tot) {
    double q = sigma_in / two_m;
    for (W t : tot) { double f = t / two_m; q -= f * f; }
    return q;
  }
};

// Community totals Sigma_c and intra-community arc weight; membership ids must be in [0, n).
template <class A>
double modularity_of(const Graph<typename A::W>& g, const int32_t* C) {
  typedef typename A::W W;
  std::vector<W> tot(g.n > 0 ? g.n : 1, W(0));
  W two_m = 0, sig = 0;
  for (int64_t i = 0; i < g.n; i++)
    for (int64_t e = g.off[i]; e < g.off[i + 1]; e++) {
      W w = g.w[e];
      two_m += w;
      tot[C[i]] += w;
      if (C[g.tg[e]] == C[i]) sig += w;
    }
  if (two_m == W(0)) return 0.0;
  return A::modularity(two_m, sig, tot);
}

// Greedy colouring in decreasing priority: colour(v) = smallest colour unused by the already
// coloured (= higher-priority) neighbours u != v.  Equals what Jones-Plassmann rounds compute.
template <class W>
int32_t colour_graph(const Graph<W>& g, uint64_t seed, int32_t pass, std::vector<int32_t>& col) {
  std::vector<std::pair<uint64_t, int32_t>> order(g.n);
  for (int64_t v = 0; v < g.n; v++) order[v] = {hash3(seed, (uint64_t)pass, (uint64_t)v), (int32_t)v};
  std::sort(order.begin(), order.end(), [](const std::pair<uint64_t, int32_t>& a, const std::pair<uint64_t, int32_t>& b) {
    return a.first != b.first ? a.first > b.first : a.second > b.second;
  });
  col.assign(g.n, -1);
  std::vector<int64_t> stamp;
  int32_t ncol = 0;
  for (int64_t r = 0; r < g.n; r++) {
    int32_t v = order[r].second;
    int64_t deg = g.off[v + 1] - g.off[v];
    if ((int64_t)stamp.size() < deg + 1) stamp.resize(deg + 1, -1);
    for (int64_t e = g.off[v]; e < g.off[v + 1]; e++) {
      int32_t u = g.tg[e];
      if (u == v || col[u] < 0) continue;
      if (col[u] <= deg) stamp[col[u]] = r;
    }
    int32_t c = 0;
    while (c <= deg && stamp[c] == r) c++;
    col[v] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  return ncol;
}

// Collision-free table over community ids (a key list plus a value per id): the scan of
// Algorithm 2's scanCommunities.
template <class W>
struct Table {
  std::vector<W> val;
  std::vector<char> has;
  std::vector<int32_t> keys;
  explicit Table(int64_t n) : val(n > 0 ? n : 1, W(0)), has(n > 0 ? n : 1, 0) {}
  void add(int32_t c, W w) {
    if (!has[c]) { has[c] = 1; keys.push_back(c); }
    val[c] += w;
  }
  void clear() {
    for (int32_t c : keys) { has[c] = 0; val[c] = W(0); }
    keys.clear();
  }
};

template <class A>
struct Mover {
  typedef typename A::W W;
  typedef typename A::S S;
  const Graph<W>& g;
  std::vector<int32_t>& Cp;
  const std::vector<W>& K;
  std::vector<W>& Sig;
  W two_m;
  Table<W> H;
  std::vector<char> flag;
  int64_t moves = 0;

  Mover(const Graph<W>& g_, std::vector<int32_t>& Cp_, const std::vector<W>& K_, std::vector<W>& Sig_, W tm)
      : g(g_), Cp(Cp_), K(K_), Sig(Sig_), two_m(tm), H(g_.n), flag(g_.n, 1) {}

  // Best community for i against the current Cp and Sig (Eq. 2 numerator, reading R2).
  bool decide(int32_t i, int32_t* c_best, W* n_best) {
    for (int64_t e = g.off[i]; e < g.off[i + 1]; e++) {
      int32_t j = g.tg[e];
      if (j == i) continue;  // scanCommunities with self = false
      H.add(Cp[j], g.w[e]);
    }
    int32_t d = Cp[i];
    W k_id = H.has[d] ? H.val[d] : W(0);
    bool found = false;
    W best = W(0);
    int32_t bc = -1;
    for (int32_t c : H.keys) {
      if (c == d) continue;
      W nscore = two_m * (H.val[c] - k_id) - K[i] * (Sig[c] - Sig[d] + K[i]);
      if (!found || nscore > best || (nscore == best && c < bc)) { found = true; best = nscore; bc = c; }
    }
    H.clear();
    *c_best = bc;
    *n_best = best;
    return found && best > W(0);
  }

  void apply(int32_t i, int32_t c, W nscore, S& sum_n, int pruning) {
    int32_t d = Cp[i];
    Sig[d] -= K[i];
    Sig[c] += K[i];
    Cp[i] = c;
    sum_n += (S)nscore;
    moves++;
    if (pruning)
      for (int64_t e = g.off[i]; e < g.off[i + 1]; e++)
        if (g.tg[e] != i) flag[g.tg[e]] = 1;
  }

  // Algorithm 2 under the colour-synchronous schedule (reading R3) or sequentially (schedule 1).
  int32_t run(const Params& p, double tau, const std::vector<int32_t>* col, int32_t ncol) {
    std::vector<std::vector<int32_t>> classes;
    if (p.schedule == 0) {
      classes.resize(ncol);
      for (int64_t v = 0; v < g.n; v++) classes[(*col)[v]].push_back((int32_t)v);
    }
    struct Dec { int32_t v, c; W n; };
    std::vector<Dec> dec;
    int32_t li = 0;
    for (int32_t it = 0; it < p.max_iterations; it++) {
      S sum_n = 0;
      if (p.schedule == 0) {
        for (int32_t k = 0; k < ncol; k++) {
          dec.clear();
          for (int32_t v : classes[k]) {
            if (p.pruning && !flag[v]) continue;
            flag[v] = 0;
            int32_t c; W ns;
            if (decide(v, &c, &ns)) dec.push_back({v, c, ns});
          }
          for (const Dec& x : dec) apply(x.v, x.c, x.n, sum_n, p.pruning);
        }
      } else {
        for (int64_t v = 0; v < g.n; v++) {
          if (p.pruning && !flag[v]) continue;
          flag[v] = 0;
          int32_t c; W ns;
          if (decide((int32_t)v, &c, &ns)) apply((int32_t)v, c, ns, sum_n, p.pruning);
        }
      }
      li = it + 1;
      if (A::converged(sum_n, two_m, tau)) break;
    }
    return li;
  }
};

template <class W>
void vertex_weights(const Graph<W>& g, std::vector<W>& K) {
  K.assign(g.n, W(0));
  for (int64_t i = 0; i < g.n; i++)
    for (int64_t e = g.off[i]; e < g.off[i + 1]; e++) K[i] += g.w[e];
}

// Rank of each occupied id among the occupied ids (reading R6); returns the count.
int64_t renumber(std::vector<int32_t>& C, int64_t id_range) {
  std::vector<int64_t> rank(id_range > 0 ? id_range : 1, 0);
  for (int32_t c : C) rank[c] = 1;
  int64_t r = 0;
  for (int64_t c = 0; c < id_range; c++) { int64_t o = rank[c]; rank[c] = r; r += o; }
  for (int32_t& c : C) c = (int32_t)rank[c];
  return r;
}

int64_t count_distinct(const std::vector<int32_t>& C, int64_t id_range) {
  std::vector<char> seen(id_range > 0 ? id_range : 1, 0);
  int64_t r = 0;
  for (int32_t c : C) if (!seen[c]) { seen[c] = 1; r++; }
  return r;
}

// Algorithm 3: community-vertex lists by counting, then per community the summed arc weight
// to every community linked to its members (scanCommunities with self = true), rows sorted.
template <class W>
Graph<W> aggregate(const Graph<W>& g, const std::vector<int32_t>& Cp, int64_t nc) {
  std::vector<int64_t> coff(nc + 1, 0);
  for (int64_t i = 0; i < g.n; i++) coff[Cp[i] + 1]++;
  for (int64_t c = 0; c < nc; c++) coff[c + 1] += coff[c];
  std::vector<int32_t> cv(g.n);
  std::vector<int64_t> cur(coff.begin(), coff.end() - 1);
  for (int64_t i = 0; i < g.n; i++) cv[cur[Cp[i]]++] = (int32_t)i;
  Graph<W> h;
  h.n = nc;
  h.off.assign(nc + 1, 0);
  Table<W> H(nc);
  for (int64_t c = 0; c < nc; c++) {
    for (int64_t k = coff[c]; k < coff[c + 1]; k++) {
      int32_t i = cv[k];
      for (int64_t e = g.off[i]; e < g.off[i + 1]; e++) H.add(Cp[g.tg[e]], g.w[e]);
    }
    std::vector<int32_t> keys = H.keys;
    std::sort(keys.begin(), keys.end());
    for (int32_t d : keys) { h.tg.push_back(d); h.w.push_back(H.val[d]); }
    h.off[c + 1] = (int64_t)h.tg.size();
    H.clear();
  }
  return h;
}

template <class W>
int validate(int64_t n, const int64_t* off, const int32_t* tg) {
  if (n < 0 || n > 0x7fffffffLL) return 1;
  if (off[0] != 0) return 1;
  for (int64_t i = 0; i < n; i++) if (off[i + 1] < off[i]) return 1;
  for (int64_t e = 0; e < off[n]; e++) if (tg[e] < 0 || tg[e] >= n) return 1;
  return 0;
}

template <class A, class WIn>
int load_graph(int64_t n, const int64_t* off, const int32_t* tg, const WIn* w, Graph<typename A::W>& g) {
  if (validate<typename A::W>(n, off, tg)) return 1;
  g.n = n;
  g.off.assign(off, off + n + 1);
  g.tg.assign(tg, tg + off[n]);
  g.w.resize(off[n]);
  double total = 0.0;
  for (int64_t e = 0; e < off[n]; e++) {
    if (!(w[e] > 0)) return 1;
    g.w[e] = (typename A::W)w[e];
    total += (double)w[e];
  }
  if (A::is_int && total >= 2147483648.0) return 3;  // 2m must stay below 2^31 (exact int64 scores)
  return 0;
}

template <class A>
int louvain(Graph<typename A::W> gp, const Params& p, int32_t* membership, double* q_out, int32_t* n_passes,
            PassStats* stats, int32_t stats_cap, const Graph<typename A::W>& g0, const int32_t* init = nullptr) {
  typedef typename A::W W;
  const int64_t n = gp.n;
  std::vector<int32_t> C(n);
  for (int64_t v = 0; v < n; v++) C[v] = (int32_t)v;
  std::vector<int32_t> Cp;
  bool pending = false;  // Cp of the last pass not yet folded into C (reading R6)
  double tau = p.tolerance;
  int32_t passes = 0;
  for (int32_t lp = 0; lp < p.max_passes; lp++) {
    std::vector<W> K, Sig;
    vertex_weights(gp, K);
    Sig = K;
    W two_m = 0;
    for (W k : K) two_m += k;
    Cp.resize(gp.n);
    for (int64_t i = 0; i < gp.n; i++) Cp[i] = (int32_t)i;
    if (lp == 0 && init) {
      // warm start (a dynamic graph's first pass): C' = the given membership, Sigma_c = the sum of
      // K_i over its members
      for (int64_t i = 0; i < gp.n; i++) Sig[i] = W(0);
      for (int64_t i = 0; i < gp.n; i++) {
        Cp[i] = init[i];
        Sig[init[i]] += K[i];
      }
    }
    std::vector<int32_t> col;
    int32_t ncol = 0;
    if (p.schedule == 0) ncol = colour_graph(gp, p.seed, lp, col);
    Mover<A> mv(gp, Cp, K, Sig, two_m);
    int32_t li = mv.run(p, tau, p.schedule == 0 ? &col : nullptr, ncol);
    pending = true;
    passes = lp + 1;
    int64_t nc = count_distinct(Cp, gp.n);
    if (stats && lp < stats_cap) {
      PassStats& s = stats[lp];
      s.pass = lp; s.iterations = li; s.moves = mv.moves; s.n_vertices = gp.n;
      s.n_arcs = (int64_t)gp.tg.size(); s.n_communities = nc;
      s.modularity = two_m == W(0) ? 0.0 : modularity_of<A>(gp, Cp.data());
    }
    if (li <= 1) break;                                                    // globally converged
    if ((double)nc / (double)gp.n > p.aggregation_tolerance) break;        // low shrink
    renumber(Cp, gp.n);
    for (int64_t v = 0; v < n; v++) C[v] = Cp[C[v]];                       // dendrogram lookup
    pending = false;
    gp = aggregate(gp, Cp, nc);
    tau /= p.tolerance_drop;                                               // threshold scaling
  }
  if (pending)
    for (int64_t v = 0; v < n; v++) C[v] = Cp[C[v]];
  renumber(C, n);
  std::copy(C.begin(), C.end(), membership);
  if (q_out) *q_out = modularity_of<A>(g0, membership);
  if (n_passes) *n_passes = passes;
  return 0;
}

}  // namespace

extern "C" {

typedef Params oracle_params;
typedef PassStats oracle_pass_stats;

uint64_t oracle_hash3(uint64_t a, uint64_t b, uint64_t c) { return hash3(a, b, c); }

/* Eq. 1 on (offsets, targets, weights) with membership ids in [0, n).  fp != 0: weights are
 * float32 and the sums are double; else int32 weights, exact integers. */
double oracle_modularity(int64_t n, const int64_t* off, const int32_t* tg, const void* w, int fp, const int32_t* C) {
  for (int64_t v = 0; v < n; v++) if (C[v] < 0 || C[v] >= n) return -2.0;
  if (fp) {
    Graph<double> g;
    if (load_graph<FpArith>(n, off, tg, (const float*)w, g)) return -2.0;
    return modularity_of<FpArith>(g, C);
  }
  Graph<int64_t> g;
  if (load_graph<IntArith>(n, off, tg, (const int32_t*)w, g)) return -2.0;
  return modularity_of<IntArith>(g, C);
}

/* Eq. 2 numerator N for moving vertex i from its community to community c (exact, int32 weights). */
int64_t oracle_move_score_int(int64_t n, const int64_t* off, const int32_t* tg, const int32_t* w, const int32_t* C,
                              int32_t i, int32_t c) {
  int64_t two_m = 0, ki = 0, kic = 0, kid = 0, sc = 0, sd = 0;
  int32_t d = C[i];
  for (int64_t v = 0; v < n; v++)
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      two_m += w[e];
      if (C[v] == c) sc += w[e];
      if (C[v] == d) sd += w[e];
    }
  for (int64_t e = off[i]; e < off[i + 1]; e++) {
    ki += w[e];
    if (tg[e] == i) continue;
    if (C[tg[e]] == c) kic += w[e];
    if (C[tg[e]] == d) kid += w[e];
  }
  return two_m * (kic - kid) - ki * (sc - sd + ki);
}

int oracle_colour(int64_t n, const int64_t* off, const int32_t* tg, uint64_t seed, int32_t pass, int32_t* colour,
                  int32_t* n_colours) {
  Graph<int64_t> g;
  if (validate<int64_t>(n, off, tg)) return 1;
  g.n = n;
  g.off.assign(off, off + n + 1);
  g.tg.assign(tg, tg + off[n]);
  std::vector<int32_t> col;
  int32_t nc = colour_graph(g, seed, pass, col);
  std::copy(col.begin(), col.end(), colour);
  *n_colours = nc;
  return 0;
}

/* Algorithm 3 for a dense membership in [0, nc): writes offsets [nc+1], rows sorted by target,
 * weights as int64 (fp == 0) or double (fp != 0) into out_w; returns the arc count, or -1 if
 * `cap` arcs do not suffice / the input is invalid. */
int64_t oracle_aggregate(int64_t n, const int64_t* off, const int32_t* tg, const void* w, int fp, const int32_t* C,
                         int64_t nc, int64_t* out_off, int32_t* out_tg, void* out_w, int64_t cap) {
  std::vector<int32_t> Cp(C, C + n);
  for (int32_t c : Cp) if (c < 0 || c >= nc) return -1;
  if (fp) {
    Graph<double> g;
    if (load_graph<FpArith>(n, off, tg, (const float*)w, g)) return -1;
    Graph<double> h = aggregate(g, Cp, nc);
    if ((int64_t)h.tg.size() > cap) return -1;
    std::copy(h.off.begin(), h.off.end(), out_off);
    std::copy(h.tg.begin(), h.tg.end(), out_tg);
    std::copy(h.w.begin(), h.w.end(), (double*)out_w);
    return (int64_t)h.tg.size();
  }
  Graph<int64_t> g;
  if (load_graph<IntArith>(n, off, tg, (const int32_t*)w, g)) return -1;
  Graph<int64_t> h = aggregate(g, Cp, nc);
  if ((int64_t)h.tg.size() > cap) return -1;
  std::copy(h.off.begin(), h.off.end(), out_off);
  std::copy(h.tg.begin(), h.tg.end(), out_tg);
  std::copy(h.w.begin(), h.w.end(), (int64_t*)out_w);
  return (int64_t)h.tg.size();
}

/* One local-moving phase (Algorithm 2) from singleton communities, colouring of pass `pass`,
 * tolerance tau.  Writes C' (not renumbered) and the iteration / move counts. */
int oracle_local_move(int64_t n, const int64_t* off, const int32_t* tg, const void* w, int fp, const oracle_params* p,
                      int32_t pass, double tau, int32_t* cp_out, int32_t* iterations, int64_t* moves) {
  if (fp) {
    Graph<double> g;
    int rc = load_graph<FpArith>(n, off, tg, (const float*)w, g);
    if (rc) return rc;
    std::vector<double> K, Sig;
    vertex_weights(g, K);
    Sig = K;
    double two_m = 0;
    for (double k : K) two_m += k;
    std::vector<int32_t> Cp(n), col;
    for (int64_t i = 0; i < n; i++) Cp[i] = (int32_t)i;
    int32_t ncol = p->schedule == 0 ? colour_graph(g, p->seed, pass, col) : 0;
    Mover<FpArith> mv(g, Cp, K, Sig, two_m);
    *iterations = mv.run(*p, tau, p->schedule == 0 ? &col : nullptr, ncol);
    *moves = mv.moves;
    std::copy(Cp.begin(), Cp.end(), cp_out);
    return 0;
  }
  Graph<int64_t> g;
  int rc = load_graph<IntArith>(n, off, tg, (const int32_t*)w, g);
  if (rc) return rc;
  std::vector<int64_t> K, Sig;
  vertex_weights(g, K);
  Sig = K;
  int64_t two_m = 0;
  for (int64_t k : K) two_m += k;
  std::vector<int32_t> Cp(n), col;
  for (int64_t i = 0; i < n; i++) Cp[i] = (int32_t)i;
  int32_t ncol = p->schedule == 0 ? colour_graph(g, p->seed, pass, col) : 0;
  Mover<IntArith> mv(g, Cp, K, Sig, two_m);
  *iterations = mv.run(*p, tau, p->schedule == 0 ? &col : nullptr, ncol);
  *moves = mv.moves;
  std::copy(Cp.begin(), Cp.end(), cp_out);
  return 0;
}

/* A batch update of a symmetric CSR with n_old rows into one with n_new >= n_old rows: every arc
 * between u and v of a deleted edge {u, v} is removed (both directions, all duplicates); then each
 * inserted edge (u, v, w) adds the arc u->v and, if u != v, the arc v->u, both of weight w.  Row r
 * of the result holds r's surviving arcs in their old order, then its inserted arcs in list order.
 * Weights int32 (fp == 0) or float32.  Returns the arc count, or -1 if an id is out of range or
 * `cap` arcs do not suffice. */
int64_t oracle_update_graph(int64_t n_old, const int64_t* off, const int32_t* tg, const void* w, int fp, int64_t n_new,
                            int64_t n_del, const int32_t* del_u, const int32_t* del_v, int64_t n_ins,
                            const int32_t* ins_u, const int32_t* ins_v, const void* ins_w, int64_t* out_off,
                            int32_t* out_tg, void* out_w, int64_t cap) {
  if (n_new < n_old || n_old < 0) return -1;
  std::vector<std::pair<int32_t, int32_t>> dels;
  for (int64_t k = 0; k < n_del; k++) {
    if (del_u[k] < 0 || del_u[k] >= n_new || del_v[k] < 0 || del_v[k] >= n_new) return -1;
    dels.push_back({std::min(del_u[k], del_v[k]), std::max(del_u[k], del_v[k])});
  }
  std::sort(dels.begin(), dels.end());
  std::vector<std::vector<std::pair<int32_t, int64_t>>> added(n_new);  // (target, insertion index)
  for (int64_t k = 0; k < n_ins; k++) {
    if (ins_u[k] < 0 || ins_u[k] >= n_new || ins_v[k] < 0 || ins_v[k] >= n_new) return -1;
    added[ins_u[k]].push_back({ins_v[k], k});
    if (ins_u[k] != ins_v[k]) added[ins_v[k]].push_back({ins_u[k], k});
  }
  int64_t a = 0;
  out_off[0] = 0;
  for (int64_t r = 0; r < n_new; r++) {
    if (r < n_old)
      for (int64_t e = off[r]; e < off[r + 1]; e++) {
        const std::pair<int32_t, int32_t> key{std::min((int32_t)r, tg[e]), std::max((int32_t)r, tg[e])};
        if (std::binary_search(dels.begin(), dels.end(), key)) continue;
        if (a >= cap) return -1;
        out_tg[a] = tg[e];
        if (fp) ((float*)out_w)[a] = ((const float*)w)[e];
        else ((int32_t*)out_w)[a] = ((const int32_t*)w)[e];
        a++;
      }
    for (const auto& x : added[r]) {
      if (a >= cap) return -1;
      out_tg[a] = x.first;
      if (fp) ((float*)out_w)[a] = ((const float*)ins_w)[x.second];
      else ((int32_t*)out_w)[a] = ((const int32_t*)ins_w)[x.second];
      a++;
    }
    out_off[r + 1] = a;
  }
  return a;
}

/* Algorithm 1 whose first pass starts from membership init[n] (ids in [0, n)) instead of
 * singletons: the warm start of a dynamic graph after a batch update.  Same returns as
 * oracle_louvain; 1 also for an id out of range. */
int oracle_louvain_from(int64_t n, const int64_t* off, const int32_t* tg, const void* w, int fp, const oracle_params* p,
                        const int32_t* init, int32_t* membership, double* q, int32_t* n_passes,
                        oracle_pass_stats* stats, int32_t stats_cap) {
  for (int64_t v = 0; v < n; v++) if (init[v] < 0 || init[v] >= n) return 1;
  if (fp) {
    Graph<double> g;
    int rc = load_graph<FpArith>(n, off, tg, (const float*)w, g);
    if (rc) return rc;
    return louvain<FpArith>(g, *p, membership, q, n_passes, stats, stats_cap, g, init);
  }
  Graph<int64_t> g;
  int rc = load_graph<IntArith>(n, off, tg, (const int32_t*)w, g);
  if (rc) return rc;
  return louvain<IntArith>(g, *p, membership, q, n_passes, stats, stats_cap, g, init);
}

/* Algorithm 1.  Returns 0 ok, 1 invalid input, 3 integer 2m >= 2^31.  membership [n] gets the
 * canonical (rank-renumbered) communities, *q the Eq. 1 modularity on the input graph. */
int oracle_louvain(int64_t n, const int64_t* off, const int32_t* tg, const void* w, int fp, const oracle_params* p,
                   int32_t* membership, double* q, int32_t* n_passes, oracle_pass_stats* stats, int32_t stats_cap) {
  if (fp) {
    Graph<double> g;
    int rc = load_graph<FpArith>(n, off, tg, (const float*)w, g);
    if (rc) return rc;
    return louvain<FpArith>(g, *p, membership, q, n_passes, stats, stats_cap, g);
  }
  Graph<int64_t> g;
  int rc = load_graph<IntArith>(n, off, tg, (const int32_t*)w, g);
  if (rc) return rc;
  return louvain<IntArith>(g, *p, membership, q, n_passes, stats, stats_cap, g);
}

}  // extern "C"
