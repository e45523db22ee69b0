// LD-Leiden oracle: a plain, sequential, slow restatement of the method.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
// loads or calls this file; only the tests, the smoke check and the
// benchmark's CPU-baseline leg do.  It shares no code, header or constant
// table with the CUDA library.
//
// What it computes, in the paper's order and notation:
//   * Eq. 1 directed weighted modularity, kept as the exact integer
//     numerator Qnum = gd*m*E - gn*P with E = sum_C e_C, P = sum_C K_C^out K_C^in
//     (Q = Qnum / (gd*m^2); gamma = gn/gd).
//   * Eq. 2 one-step gain of moving v from a to b, made exact by evaluating it
//     with a' = a \ {v} (the per-v constant the paper drops is added back):
//       G = gd*m*[w(v,b)+w(b,v)-w(v,a')-w(a',v)]
//           - gn*[k_out(K_in_b - K_in_a + k_in) + k_in(K_out_b - K_out_a + k_out)]
//     so that G == gd*m^2*(Q_after - Q_before) exactly.
//   * Sec. III-E decoupling filter: candidates by (G desc, v asc), accept
//     unless the source is already an acceptor or the target an emitter.
//   * Algorithm 1 (batch update): apply the batch, repair statistics along the
//     parent chain, InitFrontier, then N passes over levels 0..T of
//     move (<= M rounds) -> refine (<= M rounds) -> aggregate repair.
//   * Eq. 3 / Sec. III-F subtract-add aggregate repair of level r+1.
//   * Static Leiden for the initial hierarchy: the same stages from singletons
//     with every node active and a full Eq. 3 aggregation.
//
// Readings of points the paper leaves open (each also stated where used):
//   - Only adjacent communities are targets, b != a, and only G > 0 counts;
//     the argmax breaks ties to the lowest community id.
//   - Undirected graphs are symmetric matrices: an edge {i,j} is the two arcs
//     (i,j),(j,i); a self-loop is one arc.  m = sum_ij w_ij.
//   - All levels share the id space [0,n): a refined community is named by
//     its seed node, a level-(r+1) node by its refined community's id, and
//     community labels are ids too, so K_C and e_C are level independent.
//   - Expand(V) = V plus its graph neighbours; touched communities and parents
//     are recorded (they drive refinement and NextFrontier) but do not enrol
//     their members.
//   - Refinement of a batch update (TouchedRefined) is local: a node whose
//     label no longer equals its refined community's label (it moved, or took
//     its members' new label) leaves it as a singleton; the refined
//     communities that lost a node or hold an endpoint of a deleted arc are
//     split into their connected components (the seed's component keeps the
//     id, others are named by their lowest member); only singletons of the
//     reset or renamed nodes move, into refined communities adjacent to them
//     inside their own community, by the same gain with a = {v}.  The static
//     build refines from singletons.
//   - Rollback iff dQ(B) < 0; stop the move loop iff dQ(B)*alpha_inv < Q0num
//     or |V|*beta_inv < |S|; refine stops iff |V|*beta_inv < |R|; either loop
//     stops when B is empty.
//   - Pass i+1 starts with A^0 = Expand_0(level-0 nodes moved in pass i) and
//     empty upper frontiers; the passes stop when that is empty or the pass
//     gain*alpha_inv < Qnum at the pass start.
//   - A level-(r+1) node exists iff some level-r node maps to it; a new one
//     has no parent until its own level is refined; an emptied one is removed
//     from its parent.
//   - Static Leiden: one pass, move and refine use up to Mst rounds, and the
//     hierarchy stops growing when refinement merges nothing or at level L.
//
// Pins (tests/test_oracle_*.py): Eq. 1 against an O(n^2) brute-force double
// sum; the gain against brute-force recomputed modularity for every (v, b);
// the target and gain that best_move and best_ref choose (the functions the
// loops call, run on one node) against an exhaustive argmax of brute-force
// numerator changes over the admissible targets (positive gains only,
// adjacent targets only, lowest id on ties; gamma 1 and 3/2);
// the decoupling filter against its defining greedy property; the repaired
// hierarchy against a from-scratch Eq. 3 rebuild after every batch; delete
// then re-insert restoring every statistic; undirected == symmetric directed;
// refined communities connected and nested; static Leiden's closed forms
// (disjoint cliques) and the brute-force optimum on tiny graphs.
// Parity unpinned: the frontier-selection and pass-control readings
// (Expand, TouchedRefined, SPExpand, NextFrontier, the stopping tests and
// the static schedule) have no printed example in the paper; the invariants
// above hold under any such choice, so the trajectory itself is fixed only by
// this restatement.

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace {

typedef int64_t i64;
typedef __int128 i128;
const int32_t NONE = -1;

enum Status { ST_OK = 0, ST_INVALID = 1, ST_RANGE = 2, ST_NO_EDGE = 3, ST_NEG_WEIGHT = 4,
              ST_OVERFLOW = 8 };
enum Op { OP_INSERT = 0, OP_DELETE = 1, OP_REWEIGHT = 2 };

typedef std::vector<std::pair<int32_t, i64>> Row;  // sorted by neighbour id

[[noreturn]] void die(const char* msg) {
  std::fprintf(stderr, "oracle internal error: %s\n", msg);
  std::abort();
}

i64 row_get(const Row& r, int32_t c) {
  auto it = std::lower_bound(r.begin(), r.end(), std::make_pair(c, (i64)INT64_MIN));
  return (it != r.end() && it->first == c) ? it->second : 0;
}

struct Level {
  std::vector<Row> out, in;          // in: used only for directed graphs
  std::vector<i64> kout, kin;        // node strengths at this level
  std::vector<int32_t> lab;          // P^r: community label of each node
  std::vector<int32_t> par;          // pi_r: parent (level r+1 node), NONE if none
  std::vector<int32_t> cnt;          // number of level r-1 children (level 0: 1)
  std::vector<uint8_t> alive;
  std::vector<int32_t> brk;          // endpoints of arcs deleted since this level was last refined
};

struct Cand {
  int32_t v, src, dst;
  i128 g;
};

struct Counters {
  i64 moves = 0, refine_moves = 0, rollbacks = 0, rounds = 0, scanned = 0, candidates = 0,
      agg_records = 0, passes = 0;
};

struct Orc {
  i64 n = 0;
  int directed = 0;
  i64 gn = 1, gd = 1;
  int N = 2, L = 4, M = 5, Mst = 20;
  i64 ainv = 1000, binv = 100;
  int T = 0;
  std::vector<Level> lv;
  std::vector<i64> Kout, Kin, e;
  i64 m = 0;
  i128 Q = 0;
  i128 Qrep = 0;  // numerator right after the statistic repair of the last batch
  Counters ctr;
  // scratch
  std::vector<i64> acc;
  std::vector<uint8_t> acc_has;
  std::vector<int32_t> keys;
  std::vector<uint8_t> flag, flag2;
  std::vector<int32_t> oldlab;
  std::vector<int8_t> role;

  const Row& inrow(int r, int32_t v) const { return directed ? lv[r].in[v] : lv[r].out[v]; }

  void alloc_level(Level& L0) {
    L0.out.assign(n, Row());
    if (directed) L0.in.assign(n, Row());
    L0.kout.assign(n, 0);
    L0.kin.assign(n, 0);
    L0.lab.assign(n, 0);
    L0.par.assign(n, NONE);
    L0.cnt.assign(n, 0);
    L0.alive.assign(n, 0);
  }

  // Eq. 1 numerator from the community statistics.
  i128 q_from_stats() const {
    i128 q = 0;
    for (i64 c = 0; c < n; ++c) q += (i128)gd * m * e[c] - (i128)gn * Kout[c] * Kin[c];
    return q;
  }

  // ---------------------------------------------------------------- sets
  static void uniq(std::vector<int32_t>& s) {
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
  }

  // Records (key, value) grouped by key with their values summed; zero sums
  // are dropped.  Plain sort-then-merge.
  typedef std::pair<std::pair<int32_t, int32_t>, i64> ERec;
  typedef std::pair<int32_t, std::pair<i64, i64>> NRec;
  static void group(std::vector<ERec>& v) {
    std::sort(v.begin(), v.end(), [](const ERec& a, const ERec& b) { return a.first < b.first; });
    size_t k = 0;
    for (size_t i = 0; i < v.size();) {
      size_t j = i;
      i64 s = 0;
      while (j < v.size() && v[j].first == v[i].first) s += v[j++].second;
      if (s != 0) v[k++] = ERec(v[i].first, s);
      i = j;
    }
    v.resize(k);
  }
  static void group(std::vector<NRec>& v) {
    std::sort(v.begin(), v.end(), [](const NRec& a, const NRec& b) { return a.first < b.first; });
    size_t k = 0;
    for (size_t i = 0; i < v.size();) {
      size_t j = i;
      i64 a = 0, b = 0;
      while (j < v.size() && v[j].first == v[i].first) { a += v[j].second.first; b += v[j].second.second; ++j; }
      if (a != 0 || b != 0) v[k++] = NRec(v[i].first, std::make_pair(a, b));
      i = j;
    }
    v.resize(k);
  }

  // Adds grouped records (sorted by (row, col), nonzero) to the rows: each
  // touched row is merged with its records in one pass; entries that reach
  // zero disappear (their endpoints are appended to `gone` when given).
  static void merge_rows_with(std::vector<Row>& rows, const std::vector<ERec>& recs,
                              std::vector<int32_t>* gone = nullptr) {
    Row merged;
    for (size_t i = 0; i < recs.size();) {
      const int32_t x = recs[i].first.first;
      size_t j = i;
      while (j < recs.size() && recs[j].first.first == x) ++j;
      Row& row = rows[x];
      merged.clear();
      size_t a = 0, b = i;
      while (a < row.size() || b < j) {
        if (b == j || (a < row.size() && row[a].first < recs[b].first.second)) {
          merged.push_back(row[a++]);
        } else if (a == row.size() || recs[b].first.second < row[a].first) {
          if (recs[b].second < 0) die("negative weight on insert");
          merged.push_back(std::make_pair(recs[b].first.second, recs[b].second));
          ++b;
        } else {
          const i64 v = row[a].second + recs[b].second;
          if (v < 0) die("negative weight");
          if (v != 0) merged.push_back(std::make_pair(row[a].first, v));
          else if (gone) { gone->push_back(x); gone->push_back(row[a].first); }
          ++a;
          ++b;
        }
      }
      row.swap(merged);
      i = j;
    }
  }

  // Applies grouped arc records to level r (out-rows, and in-rows when
  // directed); the endpoints of arcs that disappear are recorded for the
  // level's next refinement.
  void apply_arcs(int r, const std::vector<ERec>& recs) {
    merge_rows_with(lv[r].out, recs, &lv[r].brk);
    if (directed) {
      std::vector<ERec> t;
      t.reserve(recs.size());
      for (auto& x : recs) t.push_back(ERec({x.first.second, x.first.first}, x.second));
      std::sort(t.begin(), t.end(), [](const ERec& a, const ERec& b) { return a.first < b.first; });
      merge_rows_with(lv[r].in, t);
    }
  }

  // N_r(U) together with U (out- and in-neighbours), without repeats.
  std::vector<int32_t> expand(int r, const std::vector<int32_t>& U) {
    std::vector<int32_t> S;
    auto add = [&](int32_t x) {
      if (!flag2[x]) { flag2[x] = 1; S.push_back(x); }
    };
    for (int32_t v : U) {
      add(v);
      for (auto& p : lv[r].out[v]) add(p.first);
      if (directed)
        for (auto& p : lv[r].in[v]) add(p.first);
    }
    for (int32_t x : S) flag2[x] = 0;
    return S;
  }

  // Union of two node sets given as vectors without repeats.
  void unite(std::vector<int32_t>& A, const std::vector<int32_t>& B) {
    for (int32_t x : A) flag2[x] = 1;
    for (int32_t x : B)
      if (!flag2[x]) { flag2[x] = 1; A.push_back(x); }
    for (int32_t x : A) flag2[x] = 0;
  }

  // ---------------------------------------------------------------- BestMove
  // Per node of S: the best positive exact Eq. 2 gain over adjacent
  // communities other than its own (ties to the lowest community id).
  std::vector<Cand> best_move(int r, const std::vector<int32_t>& S) {
    Level& Lr = lv[r];
    std::vector<Cand> out;
    for (int32_t v : S) {
      if (!Lr.alive[v]) continue;
      int32_t a = Lr.lab[v];
      keys.clear();
      auto gather = [&](const Row& row) {
        for (auto& p : row) {
          if (p.first == v) continue;
          int32_t c = Lr.lab[p.first];
          if (!acc_has[c]) { acc_has[c] = 1; acc[c] = 0; keys.push_back(c); }
          acc[c] += p.second;
          ctr.scanned++;
        }
      };
      gather(Lr.out[v]);
      gather(inrow(r, v));
      i64 wa = acc_has[a] ? acc[a] : 0;
      bool have = false;
      int32_t bb = 0;
      i128 bg = 0;
      const i64 ko = Lr.kout[v], ki = Lr.kin[v];
      for (int32_t b : keys) {
        if (b == a) continue;
        i128 g = (i128)gd * m * (acc[b] - wa) -
                 (i128)gn * ((i128)ko * (Kin[b] - Kin[a] + ki) + (i128)ki * (Kout[b] - Kout[a] + ko));
        if (g > 0 && (!have || g > bg || (g == bg && b < bb))) { have = true; bg = g; bb = b; }
      }
      for (int32_t c : keys) acc_has[c] = 0;
      if (have) out.push_back(Cand{v, a, bb, bg});
    }
    ctr.candidates += (i64)out.size();
    return out;
  }

  // ---------------------------------------------------------------- Decouple
  // Sec. III-E: sort by decreasing gain (node id breaks ties), then accept a
  // candidate unless its source community is already an acceptor or its
  // target already an emitter.
  std::vector<Cand> decouple(std::vector<Cand> c) {
    std::sort(c.begin(), c.end(), [](const Cand& x, const Cand& y) {
      if (x.g != y.g) return x.g > y.g;
      return x.v < y.v;
    });
    std::vector<Cand> acc_out;
    for (const Cand& x : c) {
      if (role[x.src] == 2 || role[x.dst] == 1) continue;
      role[x.src] = 1;  // emitter
      role[x.dst] = 2;  // acceptor
      acc_out.push_back(x);
    }
    for (const Cand& x : c) { role[x.src] = 0; role[x.dst] = 0; }
    return acc_out;
  }

  // ---------------------------------------------------------------- Commit
  // Apply an accepted mini-batch at level r, repair K_C and e_C additively,
  // and return the exact change of the Eq. 1 numerator.  On rollback the
  // labels and the touched communities' statistics are restored.
  struct Snap { int32_t c; i64 ko, ki, ee; };

  i128 commit_move(int r, const std::vector<Cand>& B, std::vector<Snap>& snap) {
    Level& Lr = lv[r];
    std::vector<int32_t> touched;
    for (auto& x : B) { touched.push_back(x.src); touched.push_back(x.dst); }
    uniq(touched);
    snap.clear();
    for (int32_t c : touched) snap.push_back(Snap{c, Kout[c], Kin[c], e[c]});
    for (auto& x : B) { oldlab[x.v] = x.src; flag[x.v] = 1; Lr.lab[x.v] = x.dst; }
    for (auto& x : B) {
      Kout[x.src] -= Lr.kout[x.v]; Kin[x.src] -= Lr.kin[x.v];
      Kout[x.dst] += Lr.kout[x.v]; Kin[x.dst] += Lr.kin[x.v];
    }
    // internal weight: every arc with a moved endpoint is counted once
    for (auto& x : B) {
      const int32_t v = x.v, a = x.src, b = x.dst;
      for (auto& p : Lr.out[v]) {
        int32_t u = p.first;
        int32_t cu_old = flag[u] ? oldlab[u] : Lr.lab[u];
        int32_t cu_new = Lr.lab[u];
        if (cu_old == a) e[a] -= p.second;
        if (cu_new == b) e[b] += p.second;
      }
      for (auto& p : inrow(r, v)) {
        int32_t u = p.first;
        if (flag[u]) continue;  // counted from u's out-row (or the self-loop)
        if (Lr.lab[u] == a) e[a] -= p.second;
        if (Lr.lab[u] == b) e[b] += p.second;
      }
    }
    for (auto& x : B) flag[x.v] = 0;
    i128 dq = 0;
    for (auto& s : snap) {
      int32_t c = s.c;
      dq += (i128)gd * m * (e[c] - s.ee) - (i128)gn * ((i128)Kout[c] * Kin[c] - (i128)s.ko * s.ki);
    }
    return dq;
  }

  void rollback_move(int r, const std::vector<Cand>& B, const std::vector<Snap>& snap) {
    for (auto& x : B) lv[r].lab[x.v] = x.src;
    for (auto& s : snap) { Kout[s.c] = s.ko; Kin[s.c] = s.ki; e[s.c] = s.ee; }
  }

  // ---------------------------------------------------------------- Move loop
  // The local-move loop of Algorithm 1.  Returns the union of the frontiers U (U*) and
  // appends the moved nodes to `moved`.
  std::vector<int32_t> move_loop(int r, std::vector<int32_t> U, int rounds,
                                 std::vector<int32_t>& moved) {
    const i128 Q0 = Q;
    std::vector<int32_t> Ustar(U);
    std::vector<Snap> snap;
    for (int j = 0; j < rounds; ++j) {
      if (U.empty()) break;
      ctr.rounds++;
      std::vector<int32_t> S = expand(r, U);
      std::vector<Cand> B = decouple(best_move(r, S));
      if (B.empty()) break;
      i128 dq = commit_move(r, B, snap);
      if (dq < 0) {
        rollback_move(r, B, snap);
        ctr.rollbacks++;
        break;
      }
      Q += dq;
      ctr.moves += (i64)B.size();
      std::vector<int32_t> V;
      for (auto& x : B) V.push_back(x.v);
      uniq(V);
      moved.insert(moved.end(), V.begin(), V.end());
      U = expand(r, V);
      unite(Ustar, U);
      if (dq * (i128)ainv < Q0) break;
      if ((i64)V.size() * binv < (i64)S.size()) break;
    }
    return Ustar;
  }

  // Labels of every level below r follow their parents (invariant
  // P^q(u) = P^{q+1}(pi_q(u))), after moves at level r.
  void push_down(int r) {
    for (int q = r - 1; q >= 0; --q) {
      Level& A = lv[q];
      Level& Bv = lv[q + 1];
      for (i64 u = 0; u < n; ++u)
        if (A.alive[u]) {
          if (A.par[u] == NONE) die("push_down: node without parent");
          A.lab[u] = Bv.lab[A.par[u]];
        }
    }
  }

  // ---------------------------------------------------------------- Refine
  // Static build: every alive level-r node whose refined community holds a
  // node of Ustar (plus parentless new nodes) becomes a singleton refined
  // community named by its own id (with Ustar = all nodes, refinement starts
  // from singletons).  Level r+1 strengths and child counts follow live.
  // Returns D; par_old receives old parents.
  std::vector<int32_t> dissolve(int r, const std::vector<int32_t>& Ustar,
                                std::vector<int32_t>& par_old) {
    Level& Lr = lv[r];
    Level& Ln = lv[r + 1];
    std::vector<uint8_t> touchedX(n, 0), inU(n, 0);
    for (int32_t u : Ustar) {
      inU[u] = 1;
      if (Lr.par[u] != NONE) touchedX[Lr.par[u]] = 1;
    }
    std::vector<int32_t> D;
    for (i64 u = 0; u < n; ++u) {
      if (!Lr.alive[u]) continue;
      if (Lr.par[u] == NONE) {
        if (!inU[u]) die("parentless node outside the frontier");
        D.push_back((int32_t)u);
      } else if (touchedX[Lr.par[u]]) {
        D.push_back((int32_t)u);
      }
    }
    for (int32_t u : D) {
      int32_t p = Lr.par[u];
      par_old[u] = p;
      if (p != NONE) {
        Ln.kout[p] -= Lr.kout[u];
        Ln.kin[p] -= Lr.kin[u];
        Ln.cnt[p] -= 1;
      }
    }
    for (int32_t u : D) {
      Lr.par[u] = u;
      Ln.kout[u] += Lr.kout[u];
      Ln.kin[u] += Lr.kin[u];
      Ln.cnt[u] += 1;
    }
    return D;
  }

  // TouchedRefined of a batch update at level r (Sec. III-C: refinement
  // revisits only the communities touched by accepted moves).  A refined
  // community lies inside one community, so a level-r node whose label no
  // longer equals its refined community's label (it moved at level r, or its
  // label was taken from its members' moves at level r-1) leaves it and
  // becomes a singleton named by its own id, as does a parentless new node;
  // such nodes all lie in Ustar.  Every refined community that lost a node,
  // or holds an endpoint of a level-r arc deleted since the level was last
  // refined, is re-checked for connectivity over the arcs among its remaining
  // members (a refined community stays connected): the component holding the
  // community's seed node keeps the community's id, any other component is
  // renamed after its lowest member (an id no refined community uses).
  // Untouched refined communities keep their ids and members.  Level r+1
  // strengths and child counts follow.  Returns D, every node whose refined
  // community was reset or renamed; par_old receives their old parents.
  std::vector<int32_t> split(int r, const std::vector<int32_t>& Ustar, std::vector<int32_t>& par_old) {
    Level& Lr = lv[r];
    Level& Ln = lv[r + 1];
    std::vector<uint8_t> inD(n, 0), mv(n, 0), chk(n, 0);
    std::vector<int32_t> D, CK, leave;
    auto reparent = [&](int32_t u, int32_t p) {
      const int32_t po = Lr.par[u];
      if (!inD[u]) { inD[u] = 1; par_old[u] = po; D.push_back(u); }
      if (po != NONE) { Ln.kout[po] -= Lr.kout[u]; Ln.kin[po] -= Lr.kin[u]; Ln.cnt[po] -= 1; }
      Lr.par[u] = p;
      Ln.kout[p] += Lr.kout[u]; Ln.kin[p] += Lr.kin[u]; Ln.cnt[p] += 1;
    };
    auto check_later = [&](int32_t X) {
      if (X != NONE && !chk[X]) { chk[X] = 1; CK.push_back(X); }
    };
    for (int32_t u : Ustar) {
      if (!Lr.alive[u]) continue;
      const int32_t X = Lr.par[u];
      if (X == NONE || Ln.lab[X] != Lr.lab[u]) { mv[u] = 1; leave.push_back(u); check_later(X); }
    }
    for (int32_t z : Lr.brk)
      if (Lr.alive[z]) check_later(Lr.par[z]);
    for (int32_t u : leave) reparent(u, u);
    for (i64 u = 0; u < n; ++u)
      if (Lr.alive[u] && (Lr.par[u] == NONE || Ln.lab[Lr.par[u]] != Lr.lab[u]) && !mv[u])
        die("node outside the frontier left its refined community's community");
    // remaining members of the re-checked communities, in ascending id order
    std::sort(CK.begin(), CK.end());
    std::vector<std::vector<int32_t>> mem(CK.size());
    std::vector<int32_t> slot(n, -1);
    for (size_t k = 0; k < CK.size(); ++k) slot[CK[k]] = (int32_t)k;
    for (i64 u = 0; u < n; ++u)
      if (Lr.alive[u] && !mv[u] && Lr.par[u] != NONE && slot[Lr.par[u]] >= 0) mem[slot[Lr.par[u]]].push_back((int32_t)u);
    std::vector<uint8_t> seen(n, 0);
    std::vector<int32_t> comp, stack;
    for (size_t k = 0; k < CK.size(); ++k) {
      const int32_t X = CK[k];
      const bool seed_stays = Lr.alive[X] && !mv[X] && Lr.par[X] == X;
      for (int32_t s0 : mem[k]) {
        if (seen[s0]) continue;
        // one component by depth-first search over arcs among remaining members
        comp.assign(1, s0);
        stack.assign(1, s0);
        seen[s0] = 1;
        bool has_seed = false;
        while (!stack.empty()) {
          const int32_t u = stack.back();
          stack.pop_back();
          if (u == X) has_seed = true;
          auto visit = [&](const Row& row) {
            for (auto& p : row) {
              const int32_t y = p.first;
              if (!seen[y] && !mv[y] && Lr.par[y] == X && Lr.alive[y]) {
                seen[y] = 1;
                comp.push_back(y);
                stack.push_back(y);
              }
            }
          };
          visit(Lr.out[u]);
          if (directed) visit(Lr.in[u]);
        }
        if (seed_stays && has_seed) continue;
        const int32_t name = *std::min_element(comp.begin(), comp.end());
        for (int32_t u : comp) reparent(u, name);
      }
    }
    Lr.brk.clear();
    return D;
  }

  // BestRef: a still-singleton node v moves into the adjacent refined
  // community X of its own community with the best positive gain
  //   G = gd*m*(w(v,X)+w(X,v)) - gn*(k_out(v) K_in(X) + k_in(v) K_out(X)),
  // the exact Eq. 2 gain with a = {v} over refined totals (= level r+1
  // strengths); ties go to the lowest X.
  std::vector<Cand> best_ref(int r, const std::vector<int32_t>& R) {
    Level& Lr = lv[r];
    Level& Ln = lv[r + 1];
    std::vector<Cand> out;
    for (int32_t v : R) {
      const int32_t cv = Lr.lab[v];
      keys.clear();
      auto gather = [&](const Row& row) {
        for (auto& p : row) {
          int32_t u = p.first;
          if (u == v) continue;
          ctr.scanned++;
          if (Lr.lab[u] != cv) continue;
          int32_t X = Lr.par[u];
          if (!acc_has[X]) { acc_has[X] = 1; acc[X] = 0; keys.push_back(X); }
          acc[X] += p.second;
        }
      };
      gather(Lr.out[v]);
      gather(inrow(r, v));
      bool have = false;
      int32_t bx = 0;
      i128 bg = 0;
      const i64 ko = Lr.kout[v], ki = Lr.kin[v];
      for (int32_t X : keys) {
        if (X == v) continue;
        i128 g = (i128)gd * m * acc[X] - (i128)gn * ((i128)ko * Ln.kin[X] + (i128)ki * Ln.kout[X]);
        if (g > 0 && (!have || g > bg || (g == bg && X < bx))) { have = true; bg = g; bx = X; }
      }
      for (int32_t c : keys) acc_has[c] = 0;
      if (have) out.push_back(Cand{v, v, bx, bg});
    }
    ctr.candidates += (i64)out.size();
    return out;
  }

  bool singleton(int r, int32_t v) const {
    return lv[r].par[v] == v && lv[r + 1].cnt[v] == 1;
  }

  // Refinement rounds (the refinement loop of Algorithm 1).  Returns the number of
  // merges committed.
  i64 refine_loop(int r, const std::vector<int32_t>& D, int rounds) {
    Level& Lr = lv[r];
    Level& Ln = lv[r + 1];
    std::vector<uint8_t> inD(n, 0);
    for (int32_t u : D) inD[u] = 1;
    std::vector<int32_t> R;
    for (int32_t u : D)
      if (singleton(r, u)) R.push_back(u);
    i64 merges = 0;
    for (int j = 0; j < rounds; ++j) {
      if (R.empty()) break;
      ctr.rounds++;
      std::vector<Cand> B = decouple(best_ref(r, R));
      if (B.empty()) break;
      for (auto& x : B) {
        Lr.par[x.v] = x.dst;
        Ln.kout[x.dst] += Lr.kout[x.v]; Ln.kin[x.dst] += Lr.kin[x.v];
        Ln.kout[x.v] -= Lr.kout[x.v]; Ln.kin[x.v] -= Lr.kin[x.v];
        Ln.cnt[x.dst] += 1; Ln.cnt[x.v] -= 1;
      }
      merges += (i64)B.size();
      ctr.refine_moves += (i64)B.size();
      if ((i64)B.size() * binv < (i64)R.size()) break;
      // SPExpand: dissolved, still-singleton neighbours in the same community
      std::vector<int32_t> Rn;
      for (auto& x : B) {
        int32_t v = x.v;
        auto visit = [&](const Row& row) {
          for (auto& p : row) {
            int32_t u = p.first;
            if (inD[u] && Lr.lab[u] == Lr.lab[v] && singleton(r, u)) Rn.push_back(u);
          }
        };
        visit(Lr.out[v]);
        if (directed) visit(Lr.in[v]);
      }
      uniq(Rn);
      R.swap(Rn);
    }
    return merges;
  }

  // ---------------------------------------------------------------- Aggregate
  // Eq. 3 subtract-add repair of level r+1 after the parents of D changed,
  // followed by propagation of every level-(r+1) weight and strength change
  // up the parent chain, removal of emptied nodes and relabelling of the
  // level-(r+1) images.  Returns the endpoints for NextFrontier.
  std::vector<int32_t> aggregate(int r, const std::vector<int32_t>& D,
                                 const std::vector<int32_t>& par_old,
                                 const std::vector<int32_t>& relabel_from) {
    Level& Lr = lv[r];
    std::vector<uint8_t> changed(n, 0);
    std::vector<int32_t> Dc;
    for (int32_t u : D)
      if (Lr.par[u] != par_old[u]) { changed[u] = 1; Dc.push_back(u); }
    std::vector<ERec> rec;
    std::vector<NRec> nd;
    for (int32_t u : Dc) {
      const int32_t po = par_old[u], pn = Lr.par[u];
      for (auto& p : Lr.out[u]) {
        int32_t v = p.first;
        int32_t pvo = changed[v] ? par_old[v] : Lr.par[v];
        int32_t pvn = Lr.par[v];
        if (po != NONE && pvo != NONE) rec.push_back(ERec({po, pvo}, -p.second));
        rec.push_back(ERec({pn, pvn}, p.second));
      }
      for (auto& p : inrow(r, u)) {
        int32_t v = p.first;
        if (changed[v]) continue;  // counted from v's out-row (or the self-loop)
        if (po != NONE) rec.push_back(ERec({Lr.par[v], po}, -p.second));
        rec.push_back(ERec({Lr.par[v], pn}, p.second));
      }
      if (po != NONE) nd.push_back(NRec(po, std::make_pair(-Lr.kout[u], -Lr.kin[u])));
      nd.push_back(NRec(pn, std::make_pair(Lr.kout[u], Lr.kin[u])));
    }
    group(rec);
    group(nd);
    std::vector<int32_t> ends;
    std::vector<ERec> cur(rec);
    for (auto& kv : cur) {
      ends.push_back(kv.first.first);
      ends.push_back(kv.first.second);
    }
    ctr.agg_records += (i64)cur.size();
    std::vector<NRec> curk(nd);
    for (auto& kv : curk) ends.push_back(kv.first);
    // level r+1: weights change here; strengths already follow live
    apply_arcs(r + 1, cur);
    // levels r+2..T: propagate through the current parent maps
    for (int q = r + 1; q < T; ++q) {
      std::vector<ERec> up;
      std::vector<NRec> upk;
      for (auto& x : cur) {
        int32_t a = lv[q].par[x.first.first], b = lv[q].par[x.first.second];
        if (a == NONE || b == NONE) continue;
        up.push_back(ERec({a, b}, x.second));
      }
      for (auto& x : curk) {
        int32_t a = lv[q].par[x.first];
        if (a == NONE) continue;
        upk.push_back(NRec(a, x.second));
      }
      group(up);
      group(upk);
      apply_arcs(q + 1, up);
      for (auto& kv : upk) {
        lv[q + 1].kout[kv.first] += kv.second.first;
        lv[q + 1].kin[kv.first] += kv.second.second;
      }
      cur.swap(up);
      curk.swap(upk);
    }
    // existence: new nodes appear, emptied nodes leave their parents
    for (int q = r + 1; q <= T; ++q) {
      Level& Lq = lv[q];
      for (i64 x = 0; x < n; ++x) {
        if (!Lq.alive[x] && Lq.cnt[x] > 0) {
          Lq.alive[x] = 1;
          if (Lq.par[x] != NONE && q < T) die("new node with a parent");
        } else if (Lq.alive[x] && Lq.cnt[x] == 0) {
          Lq.alive[x] = 0;
          if (Lq.kout[x] != 0 || Lq.kin[x] != 0 || !Lq.out[x].empty()) die("emptied node keeps weight");
          if (q < T && Lq.par[x] != NONE) {
            lv[q + 1].cnt[Lq.par[x]] -= 1;
            Lq.par[x] = NONE;
          }
        }
      }
    }
    // the images of changed and frontier nodes carry their members' label
    for (int32_t u : relabel_from)
      if (Lr.alive[u]) lv[r + 1].lab[Lr.par[u]] = Lr.lab[u];
    for (int32_t u : D)
      if (par_old[u] != NONE) ends.push_back(par_old[u]);
    for (int32_t u : relabel_from)
      if (Lr.alive[u]) ends.push_back(Lr.par[u]);
    std::vector<int32_t> F;
    for (int32_t x : ends)
      if (lv[r + 1].alive[x]) F.push_back(x);
    uniq(F);
    return F;
  }

  // ---------------------------------------------------------------- levels
  // Refine and aggregate level r (r < T); returns NextFrontier for r+1.
  std::vector<int32_t> refine_aggregate(int r, const std::vector<int32_t>& Ustar, int rounds, i64* merges_out) {
    std::vector<int32_t> par_old(n, NONE);
    std::vector<int32_t> D = split(r, Ustar, par_old);
    i64 merges = refine_loop(r, D, rounds);
    if (merges_out) *merges_out = merges;
    std::vector<int32_t> rel(Ustar);
    rel.insert(rel.end(), D.begin(), D.end());
    uniq(rel);
    return aggregate(r, D, par_old, rel);
  }

  // ---------------------------------------------------------------- create
  int create(i64 n_, i64 nnz, const i64* rp, const int32_t* col, const int32_t* w) {
    n = n_;
    if (n <= 0 || n > INT32_MAX) return ST_INVALID;
    if (L < 0 || L > 8 || N < 0 || M < 0 || Mst < 0 || ainv <= 0 || binv <= 0 || gn <= 0 ||
        gd <= 0 || gn > 1024 || gd > 1024)
      return ST_INVALID;
    if (rp[0] != 0 || rp[n] != nnz) return ST_INVALID;
    for (i64 v = 0; v < n; ++v)
      if (rp[v + 1] < rp[v]) return ST_INVALID;
    for (i64 k = 0; k < nnz; ++k) {
      if (col[k] < 0 || col[k] >= n) return ST_RANGE;
      if (w[k] < 1) return ST_INVALID;
    }
    lv.assign(1, Level());
    alloc_level(lv[0]);
    Level& L0 = lv[0];
    // rows collected, then sorted with repeated entries summed
    for (i64 v = 0; v < n; ++v)
      for (i64 k = rp[v]; k < rp[v + 1]; ++k) {
        L0.out[v].push_back(std::make_pair(col[k], (i64)w[k]));
        if (directed) L0.in[col[k]].push_back(std::make_pair((int32_t)v, (i64)w[k]));
      }
    auto merge_rows = [](std::vector<Row>& rows) {
      for (Row& row : rows) {
        std::sort(row.begin(), row.end());
        size_t k = 0;
        for (size_t i = 0; i < row.size();) {
          size_t j = i;
          i64 s = 0;
          while (j < row.size() && row[j].first == row[i].first) s += row[j++].second;
          row[k++] = std::make_pair(row[i].first, s);
          i = j;
        }
        row.resize(k);
      }
    };
    merge_rows(L0.out);
    if (directed) merge_rows(L0.in);
    i64 msum = 0;
    for (i64 v = 0; v < n; ++v)
      for (auto& p : L0.out[v]) {
        if (p.second > INT32_MAX) return ST_OVERFLOW;
        msum += p.second;
      }
    if (msum >= ((i64)1 << 50)) return ST_OVERFLOW;
    if (!directed)
      for (i64 v = 0; v < n; ++v)
        for (auto& p : L0.out[v])
          if (row_get(L0.out[p.first], (int32_t)v) != p.second) return ST_INVALID;
    m = msum;
    Kout.assign(n, 0); Kin.assign(n, 0); e.assign(n, 0);
    acc.assign(n, 0); acc_has.assign(n, 0); flag.assign(n, 0); flag2.assign(n, 0);
    oldlab.assign(n, 0); role.assign(n, 0);
    for (i64 v = 0; v < n; ++v)
      for (auto& p : L0.out[v]) { L0.kout[v] += p.second; L0.kin[p.first] += p.second; }
    for (i64 v = 0; v < n; ++v) {
      L0.lab[v] = (int32_t)v;
      L0.cnt[v] = 1;
      L0.alive[v] = 1;
      Kout[v] = L0.kout[v];
      Kin[v] = L0.kin[v];
      e[v] = row_get(L0.out[v], (int32_t)v);
    }
    Q = q_from_stats();
    // static Leiden: one pass over levels, every node active
    T = 0;
    for (int r = 0; r <= L; ++r) {
      std::vector<int32_t> U;
      for (i64 v = 0; v < n; ++v)
        if (lv[r].alive[v]) U.push_back((int32_t)v);
      std::vector<int32_t> moved;
      move_loop(r, U, Mst, moved);
      push_down(r);
      if (r == L) break;
      lv.push_back(Level());
      alloc_level(lv[r + 1]);
      T = r + 1;  // provisional, so that aggregation sees level r+1
      i64 merges = 0;
      std::vector<int32_t> par_old(n, NONE);
      std::vector<int32_t> D = dissolve(r, U, par_old);
      merges = refine_loop(r, D, Mst);
      if (merges == 0) {
        for (int32_t u : D) lv[r].par[u] = NONE;
        lv.pop_back();
        T = r;
        break;
      }
      aggregate(r, D, par_old, D);
    }
    for (auto& Lq : lv) Lq.brk.clear();
    return ST_OK;
  }

  // ---------------------------------------------------------------- apply
  int apply(const int32_t* upd, i64 count) {
    // validation of single updates, first failing index wins
    for (i64 k = 0; k < count; ++k) {
      int32_t i = upd[4 * k], j = upd[4 * k + 1], op = upd[4 * k + 2], w = upd[4 * k + 3];
      if (i < 0 || i >= n || j < 0 || j >= n) return ST_RANGE;
      if (op != OP_INSERT && op != OP_DELETE && op != OP_REWEIGHT) return ST_INVALID;
      if (op == OP_INSERT && w < 1) return ST_INVALID;
      if (op == OP_REWEIGHT && w < 0) return ST_NEG_WEIGHT;
    }
    // group by edge key, keeping array order inside a key
    std::map<std::pair<int32_t, int32_t>, std::vector<i64>> groups;
    for (i64 k = 0; k < count; ++k) {
      int32_t i = upd[4 * k], j = upd[4 * k + 1];
      std::pair<int32_t, int32_t> key = directed ? std::make_pair(i, j)
                                                 : std::make_pair(std::min(i, j), std::max(i, j));
      groups[key].push_back(k);
    }
    i64 err_at = INT64_MAX;
    int err = ST_OK;
    std::vector<std::pair<std::pair<int32_t, int32_t>, i64>> deltas;
    for (auto& g : groups) {
      const i64 old = row_get(lv[0].out[g.first.first], g.first.second);
      i64 cur = old;
      for (i64 k : g.second) {
        int32_t op = upd[4 * k + 2], w = upd[4 * k + 3];
        int bad = ST_OK;
        if (op == OP_INSERT) {
          cur += w;
          if (cur > INT32_MAX) bad = ST_OVERFLOW;
        } else if (op == OP_DELETE) {
          if (cur == 0) bad = ST_NO_EDGE;
          cur = 0;
        } else {
          if (cur == 0) bad = ST_NO_EDGE;
          cur = w;
        }
        if (bad != ST_OK) {
          if (k < err_at) { err_at = k; err = bad; }
          break;
        }
      }
      if (cur != old) deltas.push_back(std::make_pair(g.first, cur - old));
    }
    if (err != ST_OK) return err;
    i64 mnew = m;
    for (auto& d : deltas) mnew += (directed || d.first.first == d.first.second) ? d.second : 2 * d.second;
    if (mnew >= ((i64)1 << 50)) return ST_OVERFLOW;
    // Algorithm 1: apply the batch to level 0, S_t = changed endpoints
    for (auto& Lq : lv) Lq.brk.clear();
    std::vector<ERec> arcs;
    for (auto& d : deltas) {
      arcs.push_back(d);
      if (!directed && d.first.first != d.first.second)
        arcs.push_back(std::make_pair(std::make_pair(d.first.second, d.first.first), d.second));
    }
    std::vector<int32_t> St;
    std::sort(arcs.begin(), arcs.end(), [](const ERec& a, const ERec& b) { return a.first < b.first; });
    apply_arcs(0, arcs);
    for (auto& a : arcs) {
      St.push_back(a.first.first);
      St.push_back(a.first.second);
    }
    uniq(St);
    // repair m, degrees, community totals and the aggregate chain
    std::vector<ERec> chain(arcs);
    for (auto& a : arcs) {
      const int32_t i = a.first.first, j = a.first.second;
      const i64 d = a.second;
      m += d;
      lv[0].kout[i] += d;
      lv[0].kin[j] += d;
      const int32_t ci = lv[0].lab[i], cj = lv[0].lab[j];
      Kout[ci] += d;
      Kin[cj] += d;
      if (ci == cj) e[ci] += d;
    }
    // W_r(anc(i), anc(j)) += delta and the strengths, level by level
    for (int r = 1; r <= T; ++r) {
      std::vector<ERec> up;
      for (auto& a : chain) {
        const int32_t x = lv[r - 1].par[a.first.first], y = lv[r - 1].par[a.first.second];
        if (x == NONE || y == NONE) die("batch endpoint without ancestor");
        up.push_back(ERec({x, y}, a.second));
        lv[r].kout[x] += a.second;
        lv[r].kin[y] += a.second;
      }
      group(up);
      apply_arcs(r, up);
      chain.swap(up);
    }
    Q = q_from_stats();
    Qrep = Q;
    // InitFrontier
    std::vector<std::vector<int32_t>> A(T + 1);
    A[0] = St;
    for (int r = 1; r <= T; ++r) {
      for (int32_t v : A[r - 1]) A[r].push_back(lv[r - 1].par[v]);
      uniq(A[r]);
    }
    // the passes: per level move, push-down, refine, aggregate
    for (int pass = 0; pass < N; ++pass) {
      ctr.passes++;
      const i128 Qpass = Q;
      std::vector<int32_t> moved0;
      for (int r = 0; r <= T; ++r) {
        std::vector<int32_t> U;
        for (int32_t v : A[r])
          if (lv[r].alive[v]) U.push_back(v);
        if (U.empty()) continue;
        std::vector<int32_t> moved;
        std::vector<int32_t> Ustar = move_loop(r, U, M, moved);
        if (r == 0) moved0.insert(moved0.end(), moved.begin(), moved.end());
        if (r > 0) push_down(r);
        if (r < T) {
          std::vector<int32_t> F = refine_aggregate(r, Ustar, M, nullptr);
          A[r + 1].insert(A[r + 1].end(), F.begin(), F.end());
          uniq(A[r + 1]);
        }
      }
      uniq(moved0);
      std::vector<std::vector<int32_t>> An(T + 1);
      if (!moved0.empty()) An[0] = expand(0, moved0);
      A.swap(An);
      if (A[0].empty()) break;
      if ((Q - Qpass) * (i128)ainv < Qpass) break;
    }
    return ST_OK;
  }

  // ---------------------------------------------------------------- checks
  // Rebuild every level from level 0 and the parent maps (Eq. 3) and compare
  // with the maintained state; also checks the label invariant, the
  // community statistics and the numerator.  Returns "" when all agree.
  std::string check() const {
    char buf[256];
    for (int r = 0; r <= T; ++r) {
      const Level& Lr = lv[r];
      for (i64 v = 0; v < n; ++v) {
        if (!Lr.alive[v]) {
          if (!Lr.out[v].empty()) { std::snprintf(buf, sizeof buf, "dead node %lld has edges at level %d", (long long)v, r); return buf; }
          continue;
        }
        i64 ko = 0, ki = 0;
        for (auto& p : Lr.out[v]) ko += p.second;
        for (auto& p : inrow(r, v)) ki += p.second;
        if (ko != Lr.kout[v] || ki != Lr.kin[v]) { std::snprintf(buf, sizeof buf, "strength mismatch level %d node %lld", r, (long long)v); return buf; }
        if (r < T) {
          if (Lr.par[v] == NONE || !lv[r + 1].alive[Lr.par[v]]) { std::snprintf(buf, sizeof buf, "bad parent level %d node %lld", r, (long long)v); return buf; }
          if (lv[r + 1].lab[Lr.par[v]] != Lr.lab[v]) { std::snprintf(buf, sizeof buf, "label invariant level %d node %lld", r, (long long)v); return buf; }
        }
        if (r > 0 && (Lr.cnt[v] <= 0 || lv[r - 1].par[v] != v)) { std::snprintf(buf, sizeof buf, "seed invariant level %d node %lld", r, (long long)v); return buf; }
      }
      if (r < T) {
        std::vector<int32_t> c(n, 0);
        std::vector<std::map<int32_t, i64>> W(n);
        for (i64 v = 0; v < n; ++v) {
          if (!Lr.alive[v]) continue;
          c[Lr.par[v]]++;
          for (auto& p : Lr.out[v]) W[Lr.par[v]][Lr.par[p.first]] += p.second;
        }
        const Level& Ln = lv[r + 1];
        for (i64 x = 0; x < n; ++x) {
          if (c[x] != Ln.cnt[x] || (c[x] > 0) != (Ln.alive[x] != 0)) { std::snprintf(buf, sizeof buf, "child count level %d node %lld", r + 1, (long long)x); return buf; }
          if (W[x].size() != Ln.out[x].size()) { std::snprintf(buf, sizeof buf, "aggregate row size level %d node %lld", r + 1, (long long)x); return buf; }
          size_t k = 0;
          for (auto& kv : W[x]) {
            if (Ln.out[x][k].first != kv.first || Ln.out[x][k].second != kv.second) { std::snprintf(buf, sizeof buf, "aggregate weight level %d (%lld,%d)", r + 1, (long long)x, kv.first); return buf; }
            ++k;
          }
          if (directed) {
            for (auto& p : Ln.in[x])
              if (row_get(Ln.out[p.first], (int32_t)x) != p.second) { std::snprintf(buf, sizeof buf, "in/out mismatch level %d", r + 1); return buf; }
          }
        }
      } else {
        for (i64 v = 0; v < n; ++v)
          if (Lr.par[v] != NONE) { std::snprintf(buf, sizeof buf, "top level node %lld has a parent", (long long)v); return buf; }
      }
    }
    // community statistics from level-0 labels
    std::vector<i64> ko(n, 0), ki(n, 0), ee(n, 0);
    i64 mm = 0;
    const Level& L0 = lv[0];
    for (i64 v = 0; v < n; ++v)
      for (auto& p : L0.out[v]) {
        mm += p.second;
        ko[L0.lab[v]] += p.second;
        ki[L0.lab[p.first]] += p.second;
        if (L0.lab[v] == L0.lab[p.first]) ee[L0.lab[v]] += p.second;
      }
    if (mm != m) return "m mismatch";
    for (i64 c = 0; c < n; ++c)
      if (ko[c] != Kout[c] || ki[c] != Kin[c] || ee[c] != e[c]) { std::snprintf(buf, sizeof buf, "community stats mismatch %lld", (long long)c); return buf; }
    if (q_from_stats() != Q) return "numerator mismatch";
    return "";
  }
};

std::string g_msg;

}  // namespace

// ------------------------------------------------------------------ C entry points
extern "C" {

// params: directed, gamma_num, gamma_den, N, L, M, M_static, alpha_inv, beta_inv
void* orc_create(const int64_t* params, int64_t n, int64_t nnz, const int64_t* row_ptr,
                 const int32_t* col, const int32_t* w, int32_t* status) {
  Orc* o = new Orc();
  o->directed = (int)params[0];
  o->gn = params[1]; o->gd = params[2];
  o->N = (int)params[3]; o->L = (int)params[4]; o->M = (int)params[5]; o->Mst = (int)params[6];
  o->ainv = params[7]; o->binv = params[8];
  int st = o->create(n, nnz, row_ptr, col, w);
  *status = st;
  if (st != ST_OK) { delete o; return nullptr; }
  return o;
}

int32_t orc_apply(void* h, const int32_t* upd, int64_t count) {
  return ((Orc*)h)->apply(upd, count);
}

void orc_destroy(void* h) { delete (Orc*)h; }

int32_t orc_top(void* h) { return ((Orc*)h)->T; }

// Per-level node arrays (length n each); par is all NONE at the top level.
void orc_level(void* h, int32_t r, int32_t* lab, int32_t* par, int64_t* kout, int64_t* kin,
               int32_t* cnt, uint8_t* alive) {
  Orc* o = (Orc*)h;
  const Level& L = o->lv[r];
  for (int64_t v = 0; v < o->n; ++v) {
    lab[v] = L.lab[v]; par[v] = L.par[v]; kout[v] = L.kout[v]; kin[v] = L.kin[v];
    cnt[v] = L.cnt[v]; alive[v] = L.alive[v];
  }
}

int64_t orc_level_nnz(void* h, int32_t r) {
  Orc* o = (Orc*)h;
  int64_t s = 0;
  for (auto& row : o->lv[r].out) s += (int64_t)row.size();
  return s;
}

// Out-adjacency of level r as sorted CSR.
void orc_level_adj(void* h, int32_t r, int64_t* row_ptr, int32_t* col, int64_t* w) {
  Orc* o = (Orc*)h;
  int64_t k = 0;
  for (int64_t v = 0; v < o->n; ++v) {
    row_ptr[v] = k;
    for (auto& p : o->lv[r].out[v]) { col[k] = p.first; w[k] = p.second; ++k; }
  }
  row_ptr[o->n] = k;
}

void orc_comm(void* h, int64_t* Kout, int64_t* Kin, int64_t* e) {
  Orc* o = (Orc*)h;
  for (int64_t c = 0; c < o->n; ++c) { Kout[c] = o->Kout[c]; Kin[c] = o->Kin[c]; e[c] = o->e[c]; }
}

// m, and the Eq. 1 numerator as (hi, lo) 64-bit halves.
void orc_scalars(void* h, int64_t* m, int64_t* q_hi, uint64_t* q_lo) {
  Orc* o = (Orc*)h;
  *m = o->m;
  *q_hi = (int64_t)(o->Q >> 64);
  *q_lo = (uint64_t)o->Q;
}

void orc_q_repair(void* h, int64_t* q_hi, uint64_t* q_lo) {
  Orc* o = (Orc*)h;
  *q_hi = (int64_t)(o->Qrep >> 64);
  *q_lo = (uint64_t)o->Qrep;
}

double orc_modularity(void* h) {
  Orc* o = (Orc*)h;
  if (o->m == 0) return 0.0;
  return (double)o->Q / ((double)o->gd * (double)o->m * (double)o->m);
}

// counters: moves, refine_moves, rollbacks, rounds, scanned, candidates, agg_records, passes
void orc_counters(void* h, int64_t* out) {
  Counters& c = ((Orc*)h)->ctr;
  out[0] = c.moves; out[1] = c.refine_moves; out[2] = c.rollbacks; out[3] = c.rounds;
  out[4] = c.scanned; out[5] = c.candidates; out[6] = c.agg_records; out[7] = c.passes;
}

const char* orc_check(void* h) {
  g_msg = ((Orc*)h)->check();
  return g_msg.c_str();
}

// Exact Eq. 2 gain at level r of moving v to community b (any b != lab(v)).
void orc_gain(void* h, int32_t r, int32_t v, int32_t b, int64_t* g_hi, uint64_t* g_lo) {
  Orc* o = (Orc*)h;
  const Level& L = o->lv[r];
  const int32_t a = L.lab[v];
  i64 wa = 0, wb = 0;
  auto scan = [&](const Row& row) {
    for (auto& p : row) {
      if (p.first == v) continue;
      if (L.lab[p.first] == a) wa += p.second;
      if (L.lab[p.first] == b) wb += p.second;
    }
  };
  scan(L.out[v]);
  scan(o->inrow(r, v));
  const i64 ko = L.kout[v], ki = L.kin[v];
  i128 g = (i128)o->gd * o->m * (wb - wa) -
           (i128)o->gn * ((i128)ko * (o->Kin[b] - o->Kin[a] + ki) + (i128)ki * (o->Kout[b] - o->Kout[a] + ko));
  *g_hi = (int64_t)(g >> 64);
  *g_lo = (uint64_t)g;
}

// BestMove of the single node v at level r, computed by the same best_move
// the move loop calls (the search counters are left as they were).  Returns 1
// with the chosen target community and its exact gain, or 0 when v has no
// adjacent community with a positive gain (or is not alive).
int32_t orc_best_move(void* h, int32_t r, int32_t v, int32_t* target, int64_t* g_hi, uint64_t* g_lo) {
  Orc* o = (Orc*)h;
  if (r < 0 || r > o->T || v < 0 || v >= o->n) return -1;
  const Counters keep = o->ctr;
  std::vector<Cand> c = o->best_move(r, std::vector<int32_t>{v});
  o->ctr = keep;
  if (c.empty()) return 0;
  *target = c[0].dst;
  *g_hi = (int64_t)(c[0].g >> 64);
  *g_lo = (uint64_t)c[0].g;
  return 1;
}

// BestRef of the single node v at level r < T (v must be a singleton refined
// community), by the same best_ref the refinement loop calls.  Returns 1 with
// the target refined community and its exact gain, 0 when there is none, -1
// on bad arguments.
int32_t orc_best_ref(void* h, int32_t r, int32_t v, int32_t* target, int64_t* g_hi, uint64_t* g_lo) {
  Orc* o = (Orc*)h;
  if (r < 0 || r >= o->T || v < 0 || v >= o->n || !o->singleton(r, v)) return -1;
  const Counters keep = o->ctr;
  std::vector<Cand> c = o->best_ref(r, std::vector<int32_t>{v});
  o->ctr = keep;
  if (c.empty()) return 0;
  *target = c[0].dst;
  *g_hi = (int64_t)(c[0].g >> 64);
  *g_lo = (uint64_t)c[0].g;
  return 1;
}

// Test set-up: replaces the partition of a one-level state (T == 0) by lab
// (ids in [0, n)) and recomputes the community totals, internal weights and
// the Eq. 1 numerator from level 0.  Returns 0, or 1 when T > 0 or a label
// is out of range (nothing changed).
int32_t orc_set_partition(void* h, const int32_t* lab) {
  Orc* o = (Orc*)h;
  if (o->T != 0) return 1;
  for (int64_t v = 0; v < o->n; ++v)
    if (lab[v] < 0 || lab[v] >= o->n) return 1;
  Level& L0 = o->lv[0];
  for (int64_t v = 0; v < o->n; ++v) L0.lab[v] = lab[v];
  for (int64_t c = 0; c < o->n; ++c) { o->Kout[c] = 0; o->Kin[c] = 0; o->e[c] = 0; }
  for (int64_t v = 0; v < o->n; ++v)
    for (auto& p : L0.out[v]) {
      o->Kout[L0.lab[v]] += p.second;
      o->Kin[L0.lab[p.first]] += p.second;
      if (L0.lab[v] == L0.lab[p.first]) o->e[L0.lab[v]] += p.second;
    }
  o->Q = o->q_from_stats();
  return 0;
}

// Growth of the vertex set (Sec. II: V_t may change between batches): the
// vertices n .. n_new-1 are added isolated, each its own community and, at
// every level, its own node whose parent is the node of the same id one level
// up.  Returns 0, or 1 when n_new < n.
int32_t orc_grow(void* h, int64_t n_new) {
  Orc* o = (Orc*)h;
  if (n_new < o->n || n_new > INT32_MAX) return 1;
  const int64_t n = o->n;
  for (int r = 0; r <= o->T; ++r) {
    Level& L = o->lv[r];
    L.out.resize(n_new);
    if (o->directed) L.in.resize(n_new);
    L.kout.resize(n_new, 0);
    L.kin.resize(n_new, 0);
    L.lab.resize(n_new);
    L.par.resize(n_new);
    L.cnt.resize(n_new, 1);
    L.alive.resize(n_new, 1);
    for (int64_t v = n; v < n_new; ++v) {
      L.lab[v] = (int32_t)v;
      L.par[v] = r < o->T ? (int32_t)v : NONE;
    }
  }
  o->Kout.resize(n_new, 0);
  o->Kin.resize(n_new, 0);
  o->e.resize(n_new, 0);
  o->acc.resize(n_new, 0);
  o->acc_has.resize(n_new, 0);
  o->flag.resize(n_new, 0);
  o->flag2.resize(n_new, 0);
  o->oldlab.resize(n_new, 0);
  o->role.resize(n_new, 0);
  o->n = n_new;
  return 0;
}

// Decoupling filter on an explicit candidate list; accepted[k] = 1 or 0.
void orc_decouple(int64_t count, const int32_t* v, const int32_t* src, const int32_t* dst,
                  const int64_t* g_hi, const uint64_t* g_lo, int64_t id_space, uint8_t* accepted) {
  Orc o;
  o.n = id_space;
  o.role.assign(id_space, 0);
  std::vector<Cand> c;
  for (int64_t k = 0; k < count; ++k)
    c.push_back(Cand{v[k], src[k], dst[k], ((i128)g_hi[k] << 64) | (i128)g_lo[k]});
  std::vector<Cand> a = o.decouple(c);
  std::vector<uint8_t> acc(count, 0);
  for (int64_t k = 0; k < count; ++k) accepted[k] = 0;
  for (auto& x : a)
    for (int64_t k = 0; k < count; ++k)
      if (v[k] == x.v) accepted[k] = 1;
}

}  // extern "C"
