// Host-side planning: Givens factorisation of the relative rotation, the
// two-site gate of one Givens rotation, the basis change of the integrals and
// the Hamiltonian MPO.  Everything here runs once per state or per pair,
// outside the device hot loops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <exception>
#include <thread>

#include "internal.h"

namespace tnqe {

// ----------------------------------------------------------------------------- Eq. 11
// V J_1 J_2 ... J_K = D with J_t rotations on adjacent columns.  Rows of the
// remaining block are cleared alternately from the top (right to left: each
// rotation pushes the row's weight one column left) and from the bottom (left
// to right).  The state then receives G(J_1^T), ..., G(J_K^T), G(D) in that
// order; consecutive sweeps run in opposite directions, so the canonical
// centre only ever moves with the sweep.  A pair (x, y) of norm below 1e-14
// is rounding noise of an orthogonal matrix and gets the identity rotation.
GivensPlan givens_plan(const double* V, int N) {
  const double skip = 1e-14;
  std::vector<double> W(V, V + (size_t)N * N);
  auto rot = [&](int a, double c, double s) {
    for (int r = 0; r < N; ++r) {
      double x = W[(size_t)r * N + a], y = W[(size_t)r * N + a + 1];
      W[(size_t)r * N + a] = c * x + s * y;
      W[(size_t)r * N + a + 1] = -s * x + c * y;
    }
  };
  GivensPlan plan;
  int lo = 0, hi = N - 1;
  bool top = true;
  std::vector<size_t> pass_end;
  while (lo < hi) {
    if (top) {
      for (int col = hi; col > lo; --col) {
        int a = col - 1;
        double x = W[(size_t)lo * N + a], y = W[(size_t)lo * N + a + 1];
        double rho = std::hypot(x, y);
        double c = 1.0, s = 0.0;
        if (rho >= skip) { c = x / rho; s = y / rho; }
        rot(a, c, s);
        plan.gates.push_back({a, 0, c, s});
      }
      ++lo;
    } else {
      for (int col = lo; col < hi; ++col) {
        int a = col;
        double x = W[(size_t)hi * N + a], y = W[(size_t)hi * N + a + 1];
        double rho = std::hypot(x, y);
        double c = 1.0, s = 0.0;
        if (rho >= skip) { c = y / rho; s = -x / rho; }
        rot(a, c, s);
        plan.gates.push_back({a, 1, c, s});
      }
      --hi;
    }
    pass_end.push_back(plan.gates.size());
    top = !top;
  }
  // the last gate of every sweep but the final one hands the centre to the next sweep
  for (size_t p = 0; p + 1 < pass_end.size(); ++p) {
    Gate& g = plan.gates[pass_end[p] - 1];
    g.side = 1 - g.side;
  }
  plan.neg_site = (W[(size_t)lo * N + lo] < 0.0) ? lo : -1;
  return plan;
}

// ----------------------------------------------------------------------------- App. A3
// G(J^T) on sites (a, b = a+1): a+_{a s} -> c a+_{a s} - s a+_{b s},
// a+_{b s} -> s a+_{a s} + c a+_{b s}, vacuum fixed.  Each two-site basis state
// is a product of creation operators on the modes (a up, a dn, b up, b dn);
// the transformed product is expanded and normal-ordered term by term.
void gate_matrix(double c, double s, double* G) {
  std::memset(G, 0, sizeof(double) * 256);
  // image of mode m: two (mode, coefficient) pairs
  const int img_mode[4][2] = {{0, 2}, {1, 3}, {0, 2}, {1, 3}};
  const double img_coef[4][2] = {{c, -s}, {c, -s}, {s, c}, {s, c}};
  for (int K = 0; K < 16; ++K) {
    int ka = K >> 2, kb = K & 3;
    int occ[4], n = 0;
    if (ka & 1) occ[n++] = 0;
    if (ka & 2) occ[n++] = 1;
    if (kb & 1) occ[n++] = 2;
    if (kb & 2) occ[n++] = 3;
    for (int choice = 0; choice < (1 << n); ++choice) {
      int seq[4];
      double coef = 1.0;
      for (int i = 0; i < n; ++i) {
        int bit = (choice >> i) & 1;
        seq[i] = img_mode[occ[i]][bit];
        coef *= img_coef[occ[i]][bit];
      }
      bool dup = false;
      int inv = 0;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
          if (seq[i] == seq[j]) dup = true;
          if (seq[i] > seq[j]) ++inv;
        }
      if (dup || coef == 0.0) continue;
      int mask = 0;
      for (int i = 0; i < n; ++i) mask |= 1 << seq[i];
      int ka2 = (mask & 1) | ((mask >> 1) & 1) << 1;
      int kb2 = ((mask >> 2) & 1) | ((mask >> 3) & 1) << 1;
      int K2 = ka2 * 4 + kb2;
      G[K2 * 16 + K] += (inv & 1) ? -coef : coef;
    }
  }
}

// ----------------------------------------------------------------------------- Sec. IV B
// H in basis U: h' = U^T h U and (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd),
// one index at a time.
void rotate_integrals(const double* h1, const double* eri, const double* U, int N,
                      std::vector<double>& h_out, std::vector<double>& eri_out) {
  const size_t n = N, n2 = n * n, n3 = n2 * n, n4 = n3 * n;
  std::vector<double> t(n2, 0.0);
  h_out.assign(n2, 0.0);
  for (size_t a = 0; a < n; ++a)
    for (size_t q = 0; q < n; ++q) {
      double acc = 0.0;
      for (size_t b = 0; b < n; ++b) acc += h1[a * n + b] * U[b * n + q];
      t[a * n + q] = acc;
    }
  for (size_t p = 0; p < n; ++p)
    for (size_t q = 0; q < n; ++q) {
      double acc = 0.0;
      for (size_t a = 0; a < n; ++a) acc += U[a * n + p] * t[a * n + q];
      h_out[p * n + q] = acc;
    }
  std::vector<double> A(eri, eri + n4), B(n4);
  // transform the last index, then rotate index positions: (a b c d) -> (d' a b c)
  for (int pass = 0; pass < 4; ++pass) {
    for (size_t i = 0; i < n3; ++i) {
      const double* row = &A[i * n];
      for (size_t q = 0; q < n; ++q) {
        double acc = 0.0;
        for (size_t d = 0; d < n; ++d) acc += row[d] * U[d * n + q];
        B[q * n3 + i] = acc;   // new index first
      }
    }
    A.swap(B);
  }
  eri_out.swap(A);
}

// ----------------------------------------------------------------------------- Eq. 1 as an MPO
// Channels at bond b carry the operator string of a term on one side of the
// bond.  A term (its ladder operators stably sorted by spin-orbital position
// with the fermion sign) with k of its n operators left of bond b uses:
//   k = 0: the identity channel; k = n: the completed-H channel;
//   k = 1: a channel named by its left operator; k = 3: one named by its right
//   operator; k = 2: named by the left pair while b <= N/2, else the right pair.
// Keyed channels are shared by all terms with that string; the coefficient is
// applied at the single site where the term moves from a left-named to a
// right-named channel.  The local operator of a term at site t is the ordered
// product of its ladder matrices there times parity^(operators right of t).
namespace {

// local basis k = n_a + 2 n_b with |3> = a+_a a+_b |vac>
struct Mat4 { double m[16]; };
Mat4 mat_identity() { Mat4 r{}; for (int i = 0; i < 4; ++i) r.m[i * 5] = 1.0; return r; }
Mat4 mat_parity() { Mat4 r{}; r.m[0] = 1; r.m[5] = -1; r.m[10] = -1; r.m[15] = 1; return r; }
Mat4 mat_ladder(int spin, bool create) {
  Mat4 r{};
  if (spin == 0) {            // a+_alpha: |0> -> |1>, |2> -> |3>
    r.m[1 * 4 + 0] = 1.0;
    r.m[3 * 4 + 2] = 1.0;
  } else {                    // a+_beta: |0> -> |2>, |1> -> -|3>
    r.m[2 * 4 + 0] = 1.0;
    r.m[3 * 4 + 1] = -1.0;
  }
  if (!create) {
    Mat4 t{};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t.m[i * 4 + j] = r.m[j * 4 + i];
    return t;
  }
  return r;
}
Mat4 mat_mul(const Mat4& a, const Mat4& b) {
  Mat4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += a.m[i * 4 + k] * b.m[k * 4 + j];
      r.m[i * 4 + j] = acc;
    }
  return r;
}

// op code = pos * 2 + create, pos = 2 p + spin
constexpr uint64_t KEY_I = 0, KEY_F = 1;
uint64_t make_key(int type, const int* codes, int n) {
  uint64_t k = (uint64_t)type | ((uint64_t)n << 2);
  for (int i = 0; i < n; ++i) k |= (uint64_t)(codes[i] + 1) << (8 + 8 * i);
  return k;
}
int key_type(uint64_t k) { return (int)(k & 3); }   // 0 I, 1 F, 2 left-named, 3 right-named
int key_nops(uint64_t k) { return (int)((k >> 2) & 3); }

struct Block { Mat4 M; };

// Open-addressing hash map uint64 -> int (linear probing, power-of-two table)
// for the MPO builder, which looks up several keys per Hamiltonian term
// (O(N^4) terms).  No key used here has all bits set, so that value marks an
// empty slot.
class FlatMap {
 public:
  explicit FlatMap(size_t expect = 64) { rehash(std::max<size_t>(64, expect * 2)); }
  int* find(uint64_t k) {
    size_t i = slot(k);
    while (true) {
      if (keys_[i] == k) return &vals_[i];
      if (keys_[i] == EMPTY) return nullptr;
      i = (i + 1) & mask_;
    }
  }
  void insert(uint64_t k, int v) {           // k must be absent
    if (2 * (n_ + 1) > keys_.size()) rehash(keys_.size() * 2);
    size_t i = slot(k);
    while (keys_[i] != EMPTY) i = (i + 1) & mask_;
    keys_[i] = k;
    vals_[i] = v;
    ++n_;
  }
  bool contains(uint64_t k) { return find(k) != nullptr; }

 private:
  static constexpr uint64_t EMPTY = ~0ull;
  size_t slot(uint64_t k) const {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (size_t)k & mask_;
  }
  void rehash(size_t cap) {
    std::vector<uint64_t> ok;
    std::vector<int> ov;
    ok.swap(keys_);
    ov.swap(vals_);
    keys_.assign(cap, EMPTY);
    vals_.assign(cap, 0);
    mask_ = cap - 1;
    n_ = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != EMPTY) insert(ok[i], ov[i]);
  }
  std::vector<uint64_t> keys_;
  std::vector<int> vals_;
  size_t mask_ = 0, n_ = 0;
};

// Operator-string bookkeeping of a share of the Hamiltonian terms: channel
// keys seen (with the first and last bond each is alive on) and, per site, the
// 4 x 4 blocks between channel keys.  Blocks that complete a term (from the
// identity or a left-named channel into a right-named or the full one) sum the
// coefficients; the others are fixed by their keys.
struct TermSink {
  int N, half;
  const std::vector<Mat4>* lprod;
  FlatMap key_id{4096};
  std::vector<uint64_t> keys;
  std::vector<int> kstart, kend;
  std::vector<FlatMap> site_blocks;
  std::vector<std::vector<std::pair<uint64_t, Mat4>>> blocks;   // (kin_id << 32 | kout_id, M)

  TermSink(int n_sites, const std::vector<Mat4>* lp)
      : N(n_sites), half(n_sites / 2), lprod(lp), site_blocks(n_sites, FlatMap(1024)), blocks(n_sites) {
    kid(KEY_I);
    kid(KEY_F);
  }
  int kid(uint64_t k) {
    if (int* f = key_id.find(k)) return *f;
    int id = (int)keys.size();
    key_id.insert(k, id);
    keys.push_back(k);
    kstart.push_back(1 << 30);
    kend.push_back(-1);
    return id;
  }
  uint64_t key_at(const int* codes, const int* sites, int n, int b) const {
    int k = 0;
    while (k < n && sites[k] < b) ++k;
    if (k == 0) return KEY_I;
    if (k == n) return KEY_F;
    if (k == 1) return make_key(2, codes, 1);
    if (k == 3) return make_key(3, codes + 3, 1);
    return (b <= half) ? make_key(2, codes, 2) : make_key(3, codes + 2, 2);
  }
  void add_term(double coef, int n, const int* pos_in, const int* cre_in) {
    if (coef == 0.0) return;
    // identical operators (same position and kind) make the term vanish
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (pos_in[i] == pos_in[j] && cre_in[i] == cre_in[j]) return;
    int order[4];
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order, order + n, [&](int x, int y) { return pos_in[x] < pos_in[y]; });
    int inv = 0;
    for (int x = 0; x < n; ++x)
      for (int y = x + 1; y < n; ++y)
        if (order[x] > order[y] && pos_in[order[x]] != pos_in[order[y]]) ++inv;
    const double sgn = (inv & 1) ? -1.0 : 1.0;
    int codes[4], sites[4], pos[4], cre[4];
    for (int i = 0; i < n; ++i) {
      pos[i] = pos_in[order[i]];
      cre[i] = cre_in[order[i]];
      codes[i] = pos[i] * 2 + cre[i];
      sites[i] = pos[i] / 2;
    }
    // event sites: operator sites and the centre hand-over
    int ev[5], nev = 0;
    for (int i = 0; i < n; ++i)
      if (nev == 0 || ev[nev - 1] != sites[i]) ev[nev++] = sites[i];
    {
      uint64_t a = key_at(codes, sites, n, half), b = key_at(codes, sites, n, half + 1);
      bool has = false;
      for (int e = 0; e < nev; ++e) has |= (ev[e] == half);
      if (a != b && !has && half < N) {
        ev[nev++] = half;
        std::sort(ev, ev + nev);
      }
    }
    for (int e = 0; e < nev; ++e) {
      const int t = ev[e];
      int after = 0, cnt = 0, combo = 0;
      for (int i = 0; i < n; ++i) {
        if (sites[i] == t) {
          combo = combo * 4 + (pos[i] & 1) * 2 + cre[i];
          ++cnt;
        }
        if (sites[i] > t) ++after;
      }
      Mat4 M = lprod[cnt][combo];
      if (after & 1)                             // times the parity string: columns 1, 2 change sign
        for (int k = 0; k < 4; ++k) {
          M.m[k * 4 + 1] = -M.m[k * 4 + 1];
          M.m[k * 4 + 2] = -M.m[k * 4 + 2];
        }
      uint64_t kin = key_at(codes, sites, n, t), kout = key_at(codes, sites, n, t + 1);
      int iin = kid(kin), iout = kid(kout);
      kend[iin] = std::max(kend[iin], t);
      kstart[iout] = std::min(kstart[iout], t + 1);
      const bool trans = (key_type(kin) == 0 || key_type(kin) == 2) && (key_type(kout) == 1 || key_type(kout) == 3);
      const uint64_t pk = ((uint64_t)iin << 32) | (uint64_t)iout;
      int* it = site_blocks[t].find(pk);
      if (trans) {
        const double f = coef * sgn;
        if (!it) {
          Mat4 S{};
          for (int q = 0; q < 16; ++q) S.m[q] = f * M.m[q];
          site_blocks[t].insert(pk, (int)blocks[t].size());
          blocks[t].push_back({pk, S});
        } else {
          Mat4& S = blocks[t][*it].second;
          for (int q = 0; q < 16; ++q) S.m[q] += f * M.m[q];
        }
      } else if (!it) {
        site_blocks[t].insert(pk, (int)blocks[t].size());
        blocks[t].push_back({pk, M});
      }
    }
  }
  // channel keys of another sink: their ids here, alive ranges widened
  std::vector<int> merge_keys(const TermSink& o) {
    std::vector<int> gid(o.keys.size());
    for (size_t id = 0; id < o.keys.size(); ++id) {
      const int g = kid(o.keys[id]);
      gid[id] = g;
      kstart[g] = std::min(kstart[g], o.kstart[id]);
      kend[g] = std::max(kend[g], o.kend[id]);
    }
    return gid;
  }
};

// Fixed number of term shares: the MPO comes out the same on every machine.
constexpr int MPO_THREADS = 8;

// partition of a block key among the merge tasks of one site
constexpr int MERGE_PARTS = 8;
inline int part_of(uint64_t pk) { return (int)(((pk * 0x9e3779b97f4a7c15ull) >> 40) % MERGE_PARTS); }

// f(i) for i in [0, n) on MPO_THREADS threads (strided); the first exception is rethrown
template <class F>
void parallel_for(int n, F f) {
  const int nt = std::min(MPO_THREADS, std::max(1, n));
  std::vector<std::exception_ptr> errs(nt);
  auto run = [&](int w) {
    try {
      for (int i = w; i < n; i += nt) f(i);
    } catch (...) {
      errs[w] = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nt; ++w) th.emplace_back(run, w);
  run(0);
  for (auto& x : th) x.join();
  for (auto& e : errs)
    if (e) std::rethrow_exception(e);
}

}  // namespace

Mpo build_mpo(const double* h1, const double* eri, int N) {
  const int half = N / 2;
  const Mat4 I4 = mat_identity(), P4 = mat_parity();
  Mat4 lad[2][2];
  for (int sp = 0; sp < 2; ++sp)
    for (int cr = 0; cr < 2; ++cr) lad[sp][cr] = mat_ladder(sp, cr != 0);
  // products of up to four ladder operators on one site, indexed by their
  // count and (spin, create) codes in order: lprod[cnt][combo]
  std::vector<Mat4> lprod_all[5];
  lprod_all[0].assign(1, I4);
  for (int cnt = 1; cnt <= 4; ++cnt) {
    lprod_all[cnt].resize((size_t)1 << (2 * cnt));
    for (size_t combo = 0; combo < lprod_all[cnt].size(); ++combo) {
      const int last = (int)(combo & 3);
      lprod_all[cnt][combo] = mat_mul(lprod_all[cnt - 1][combo >> 2], lad[last >> 1][last & 1]);
    }
  }
  // the terms in MPO_THREADS shares (by the first index of the two-body terms),
  // each on its own thread, merged in share order
  const int nsh = std::min(MPO_THREADS, std::max(1, N));
  std::vector<TermSink> sinks;
  sinks.reserve(nsh);
  for (int w = 0; w < nsh; ++w) sinks.emplace_back(N, lprod_all);
  parallel_for(nsh, [&](int w) {
    TermSink& S = sinks[w];
    if (w == 0)
      for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q)
          for (int s = 0; s < 2; ++s) {
            int pos[2] = {2 * p + s, 2 * q + s}, cre[2] = {1, 0};
            S.add_term(h1[(size_t)p * N + q], 2, pos, cre);
          }
    // (pq|rs) with spins (s, t) and (rs|pq) with (t, s) are the same operator
    // string with the same sign (the two creators and the two annihilators
    // swap): one term with the summed coefficient per pair P = (p, q) <= R = (r, s)
    const size_t NN = (size_t)N * N;
    for (int p = w; p < N; p += nsh)
      for (int q = 0; q < N; ++q) {
        const size_t P = (size_t)p * N + q;
        for (size_t R = P; R < NN; ++R) {
          const int r = (int)(R / N), ss = (int)(R % N);
          const double vpr = eri[P * NN + R], vrp = eri[R * NN + P];
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              double coef;
              if (R != P) coef = 0.5 * vpr + 0.5 * vrp;
              else if (s == t) coef = 0.5 * vpr;
              else if (s < t) coef = vpr;                // (s, t) and (t, s) are one string
              else continue;
              if (coef == 0.0) continue;
              int pos[4] = {2 * p + s, 2 * r + t, 2 * ss + t, 2 * q + s}, cre[4] = {1, 1, 0, 0};
              S.add_term(coef, 4, pos, cre);
            }
        }
      }
  });
  TermSink& G = sinks[0];
  std::vector<std::vector<int>> gids(nsh);
  gids[0].resize(G.keys.size());
  for (size_t id = 0; id < G.keys.size(); ++id) gids[0][id] = (int)id;
  for (int w = 1; w < nsh; ++w) gids[w] = G.merge_keys(sinks[w]);
  // blocks of all shares, one task per (site, key partition): every task scans
  // the site's blocks share by share and keeps its partition, so the sums of
  // completing blocks run in share order whatever the thread timing
  std::vector<std::vector<std::pair<uint64_t, Mat4>>> pblocks((size_t)N * MERGE_PARTS);
  std::vector<FlatMap> pmap((size_t)N * MERGE_PARTS, FlatMap(256));
  parallel_for(N * MERGE_PARTS, [&](int task) {
    const int t = task / MERGE_PARTS, q = task % MERGE_PARTS;
    std::vector<std::pair<uint64_t, Mat4>>& out = pblocks[task];
    FlatMap& m = pmap[task];
    for (int w = 0; w < nsh; ++w) {
      const std::vector<int>& gid = gids[w];
      for (const auto& bl : sinks[w].blocks[t]) {
        const int iin = gid[bl.first >> 32], iout = gid[bl.first & 0xffffffffu];
        const uint64_t pk = ((uint64_t)iin << 32) | (uint64_t)iout;
        if (part_of(pk) != q) continue;
        int* it = m.find(pk);
        if (!it) {
          m.insert(pk, (int)out.size());
          out.push_back({pk, bl.second});
        } else {
          const uint64_t kin = G.keys[iin], kout = G.keys[iout];
          const bool trans = (key_type(kin) == 0 || key_type(kin) == 2) && (key_type(kout) == 1 || key_type(kout) == 3);
          if (trans) {
            Mat4& S = out[*it].second;
            for (int z = 0; z < 16; ++z) S.m[z] += bl.second.m[z];
          }
        }
      }
    }
  });
  std::vector<uint64_t>& keys = G.keys;
  std::vector<int>& kstart = G.kstart;
  std::vector<int>& kend = G.kend;
  // identity string everywhere (gives the overlap), completed H to the end
  kstart[0] = 0;
  kend[0] = N;
  kend[1] = N;
  // channel numbering per bond
  Mpo mpo;
  mpo.dims.assign(N + 1, 0);
  std::vector<std::vector<int>> chan_of(N + 1);      // key id -> channel at bond b
  for (int b = 0; b <= N; ++b) {
    std::vector<std::pair<uint64_t, int>> alive;
    for (size_t id = 2; id < keys.size(); ++id)
      if (kstart[id] <= b && b <= kend[id]) alive.push_back({keys[id], (int)id});
    std::sort(alive.begin(), alive.end());
    chan_of[b].assign(keys.size(), -1);
    int c = 0;
    chan_of[b][0] = c++;
    if (kstart[1] <= b && b <= kend[1]) chan_of[b][1] = c++;
    for (auto& a : alive) chan_of[b][a.second] = c++;
    mpo.dims[b] = c;
  }
  // per site (independent, in parallel): pass-through of every channel alive on
  // both sides of the site, then the CSR rows (counted, filled, each row sorted)
  mpo.sites.resize(N);
  parallel_for(N, [&](int t) {
    std::vector<std::pair<uint64_t, Mat4>> extra;
    for (size_t id = 0; id < keys.size(); ++id) {
      if (chan_of[t][id] < 0 || chan_of[t + 1][id] < 0) continue;
      const uint64_t pk = ((uint64_t)id << 32) | (uint64_t)id;
      if (pmap[(size_t)t * MERGE_PARTS + part_of(pk)].contains(pk)) continue;
      const int tp = key_type(keys[id]);
      const bool odd = (tp >= 2) && (key_nops(keys[id]) & 1);
      extra.push_back({pk, odd ? P4 : I4});
    }
    MpoSite& S = mpo.sites[t];
    S.Din = mpo.dims[t];
    S.Dout = mpo.dims[t + 1];
    const int nrow = 4 * S.Dout;
    S.rowptr.assign(nrow + 1, 0);
    auto each_entry = [&](auto&& f) {
      auto visit = [&](const std::pair<uint64_t, Mat4>& bl) {
        const int iin = (int)(bl.first >> 32), iout = (int)(bl.first & 0xffffffffu);
        const int w = chan_of[t][iin], wo = chan_of[t + 1][iout];
        if (w < 0 || wo < 0) throw std::runtime_error("MPO channel bookkeeping failed");
        for (int k = 0; k < 4; ++k)
          for (int kp = 0; kp < 4; ++kp) {
            const double v = bl.second.m[k * 4 + kp];
            if (v != 0.0) f(k * S.Dout + wo, w * 4 + kp, v);
          }
      };
      for (int q = 0; q < MERGE_PARTS; ++q)
        for (const auto& bl : pblocks[(size_t)t * MERGE_PARTS + q]) visit(bl);
      for (const auto& bl : extra) visit(bl);
    };
    each_entry([&](int r, int, double) { ++S.rowptr[r + 1]; });
    for (int r = 0; r < nrow; ++r) S.rowptr[r + 1] += S.rowptr[r];
    const int nz = S.rowptr[nrow];
    std::vector<std::pair<int, double>> ent(nz);
    std::vector<int> cur(S.rowptr.begin(), S.rowptr.end() - 1);
    each_entry([&](int r, int c, double v) { ent[cur[r]++] = {c, v}; });
    for (int r = 0; r < nrow; ++r) std::sort(ent.begin() + S.rowptr[r], ent.begin() + S.rowptr[r + 1]);
    S.col.resize(nz);
    S.val.resize(nz);
    for (int e = 0; e < nz; ++e) {
      S.col[e] = ent[e].first;
      S.val[e] = ent[e].second;
    }
  });
  return mpo;
}

}  // namespace tnqe
