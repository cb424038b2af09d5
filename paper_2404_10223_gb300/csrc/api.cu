// C ABI (include/tnqe.h): context, validation, host planning, device memory and
// the launch sequence of the matrix-element path.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <future>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/tnqe.h"
#include "internal.h"
#include "oz_gemm.cuh"
#include "tc_gemm.cuh"

using namespace tnqe;

namespace {

struct Error : std::runtime_error {
  tnqe_status st;
  Error(tnqe_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      throw Error(e_ == cudaErrorMemoryAllocation ? TNQE_ERR_NOMEM : TNQE_ERR_CUDA,                    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                               \
  } while (0)
#define CKL(call)                                                                                     \
  do {                                                                                                \
    int e_ = (call);                                                                                  \
    if (e_ != 0) throw Error(TNQE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString((cudaError_t)e_)); \
  } while (0)

// Bumped by every (re)allocation of a workspace buffer: a captured CUDA graph
// holds raw workspace addresses and is only replayed while this is unchanged.
std::atomic<unsigned long long> g_alloc_epoch{0};

// device allocation that grows on demand and is kept for reuse
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  void ensure(size_t bytes) {
    if (bytes <= cap) return;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t b = std::max<size_t>(bytes, 256);
    CK(cudaMalloc(&p, b));
    cap = b;
    ++g_alloc_epoch;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Arrays packed back to back at 256-byte aligned offsets, for one upload.
struct HostPack {
  std::vector<unsigned char> h;
  template <class T> size_t add(const std::vector<T>& v) {
    const size_t o = (h.size() + 255) & ~(size_t)255;
    const size_t n = v.size() * sizeof(T);
    h.resize(o + std::max<size_t>(n, 16), 0);
    if (n) std::memcpy(h.data() + o, v.data(), n);
    return o;
  }
};

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

struct DevMps {
  std::vector<int> dims;                 // N + 1
  std::vector<SectorTable> sec;          // N + 1
  std::vector<long long> off;            // N
  std::vector<double> U;
  int chi = 1;
  double* d_t = nullptr;
  long long* d_off = nullptr;
  int* d_dims = nullptr;
  SectorTable* d_sec = nullptr;
  Mpo mpo;                               // host copy (dims, CSR)
  std::vector<int*> d_rowptr, d_col, d_rowperm;
  std::vector<double*> d_val;
  std::vector<float*> d_val32;
  std::vector<float2*> d_valdf;          // (hi, lo) FP32 pairs of the MPO values
  std::vector<float4*> d_ent;            // (hi, lo, column bits, 0) per MPO nonzero
  std::vector<BsChannels> bs_ch;         // N + 1: channel classes by charge change (device pointers)
  std::vector<BsRows> bs_rows;           // N: MPO rows by charge class (device pointers)
  std::shared_future<std::shared_ptr<struct MpoPack>> mpo_future;   // the MPO's host build (add_mps)
  bool mpo_ready = false;                // the MPO is on the device and mpo holds its host copy
  std::vector<void*> owned;
  void free_all() {
    if (mpo_future.valid()) mpo_future.wait();   // the build reads this state's U
    for (void* p : owned) cudaFree(p);
    owned.clear();
  }
};

// Charge change d(w) = (d_alpha, d_beta) of every MPO channel: the charge that the
// operator string of channel w adds to the left part of a state.  Propagated
// from bond 0 (identity string, no change) through the nonzeros W[(k, w'), (w, k')],
// which set d(w') = d(w) + q(k) - q(k'); channels the forward pass does not reach
// take theirs from the right.  Every nonzero is then checked against the rule.
struct BlockTables {
  std::vector<std::vector<int>> ch_off, ch_d, ch_w;           // per bond
  std::vector<std::vector<int>> rc_off, rc_d, rc_rows, rc_nnz; // per site
};

BlockTables block_tables(const Mpo& mpo, int N) {
  const int UNSET = 1 << 20;
  std::vector<std::vector<int>> da(N + 1), db(N + 1);
  for (int b = 0; b <= N; ++b) {
    da[b].assign(mpo.dims[b], UNSET);
    db[b].assign(mpo.dims[b], UNSET);
  }
  da[0][0] = db[0][0] = 0;
  auto qa = [](int k) { return k & 1; };
  auto qb = [](int k) { return k >> 1; };
  for (int t = 0; t < N; ++t) {
    const MpoSite& S = mpo.sites[t];
    for (int row = 0; row < 4 * S.Dout; ++row) {
      const int k = row / S.Dout, wp = row % S.Dout;
      for (int e = S.rowptr[row]; e < S.rowptr[row + 1]; ++e) {
        const int w = S.col[e] / 4, kp = S.col[e] % 4;
        if (da[t][w] == UNSET || da[t + 1][wp] != UNSET) continue;
        da[t + 1][wp] = da[t][w] + qa(k) - qa(kp);
        db[t + 1][wp] = db[t][w] + qb(k) - qb(kp);
      }
    }
  }
  for (int t = N - 1; t >= 0; --t) {
    const MpoSite& S = mpo.sites[t];
    for (int row = 0; row < 4 * S.Dout; ++row) {
      const int k = row / S.Dout, wp = row % S.Dout;
      for (int e = S.rowptr[row]; e < S.rowptr[row + 1]; ++e) {
        const int w = S.col[e] / 4, kp = S.col[e] % 4;
        if (da[t][w] != UNSET || da[t + 1][wp] == UNSET) continue;
        da[t][w] = da[t + 1][wp] - qa(k) + qa(kp);
        db[t][w] = db[t + 1][wp] - qb(k) + qb(kp);
      }
    }
  }
  for (int b = 0; b <= N; ++b)
    for (int w = 0; w < mpo.dims[b]; ++w)
      if (da[b][w] == UNSET) da[b][w] = db[b][w] = 0;         // a channel no nonzero touches
  BlockTables T;
  T.ch_off.resize(N + 1);
  T.ch_d.resize(N + 1);
  T.ch_w.resize(N + 1);
  for (int b = 0; b <= N; ++b) {
    std::map<std::pair<int, int>, std::vector<int>> cls;
    for (int w = 0; w < mpo.dims[b]; ++w) cls[{da[b][w], db[b][w]}].push_back(w);
    T.ch_off[b].push_back(0);
    for (const auto& kv : cls) {
      T.ch_d[b].push_back(kv.first.first);
      T.ch_d[b].push_back(kv.first.second);
      T.ch_w[b].insert(T.ch_w[b].end(), kv.second.begin(), kv.second.end());
      T.ch_off[b].push_back((int)T.ch_w[b].size());
    }
  }
  T.rc_off.resize(N);
  T.rc_d.resize(N);
  T.rc_rows.resize(N);
  T.rc_nnz.resize(N);
  for (int t = 0; t < N; ++t) {
    const MpoSite& S = mpo.sites[t];
    std::map<std::pair<int, int>, std::vector<int>> cls;
    for (int row = 0; row < 4 * S.Dout; ++row) {
      const int k = row / S.Dout, wp = row % S.Dout;
      const int rda = da[t + 1][wp] - qa(k), rdb = db[t + 1][wp] - qb(k);
      for (int e = S.rowptr[row]; e < S.rowptr[row + 1]; ++e) {
        const int w = S.col[e] / 4, kp = S.col[e] % 4;
        if (da[t][w] - qa(kp) != rda || db[t][w] - qb(kp) != rdb)
          throw Error(TNQE_ERR_STATE, "MPO nonzero breaks particle-number conservation at site " + std::to_string(t));
      }
      cls[{rda, rdb}].push_back(row);
    }
    if ((int)cls.size() > BS_MAXRC) throw Error(TNQE_ERR_STATE, "too many MPO row charge classes");
    T.rc_off[t].push_back(0);
    for (auto& kv : cls) {
      std::vector<int>& rows = kv.second;
      std::stable_sort(rows.begin(), rows.end(), [&](int x, int y) {
        return S.rowptr[x + 1] - S.rowptr[x] > S.rowptr[y + 1] - S.rowptr[y];
      });
      int nz = 0;
      for (int r : rows) nz += S.rowptr[r + 1] - S.rowptr[r];
      T.rc_d[t].push_back(kv.first.first);
      T.rc_d[t].push_back(kv.first.second);
      T.rc_rows[t].insert(T.rc_rows[t].end(), rows.begin(), rows.end());
      T.rc_off[t].push_back((int)T.rc_rows[t].size());
      T.rc_nnz[t].push_back(nz);
    }
  }
  return T;
}

struct PairPlan {                        // cached per (i, j): Givens gates on the device (in a plan arena)
  int ngates = 0, neg_site = -1;
  double* d_gates = nullptr;
  int* d_site = nullptr;
  int* d_side = nullptr;
};

// A host-to-device copy that a graph replay repeats before launching the graph.
struct Upload {
  void* dst;
  std::vector<unsigned char> data;
};

// What the host reads back after the work of one matrix-element call has run.
struct FinishInfo {
  const unsigned char* rot_small = nullptr;   // per-pair status / FLOP records of the rotation
  size_t per_small = 0, o_stat = 0, o_flops = 0;
  int nrot = 0;
  std::vector<std::array<int, 3>> ev_reads;   // (event a, event b, profile slot): slot += elapsed(a, b)
  std::vector<double> pstat;                  // profile values known at planning time
  int launches = 0;
  bool check_err = false;
  bool single_wave = true;                    // false: the call synchronised between workspace waves
  int waves = 1;                              // workspace waves of the largest contraction of the call
  std::vector<const double*> bs_flops;        // device FLOP counters (stages 1, 2, 3) of the block-sparse form
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::vector<Upload> uploads;
  unsigned long long epoch = 0;
  FinishInfo fin;
  ~GraphEntry() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace

struct tnqe_ctx {
  tnqe_options opt{};
  int N = 0, na = 0, nb = 0;
  std::vector<double> h1, eri;
  std::vector<int> exact_dim;            // N + 1: full sector-space dimension per bond
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* stage = nullptr;                 // pinned staging of tnqe_add_mps (stage_cap doubles)
  size_t stage_cap = 0;
  std::vector<std::unique_ptr<DevMps>> mps;
  std::map<std::pair<int, int>, std::unique_ptr<PairPlan>> plans;
  std::vector<void*> plan_arenas;        // device memory of the plans, one allocation per batch
  std::string err;
  // rotation workspace
  DBuf rot_work, rot_scratch, rot_meta, rot_small, rot_desc;
  // contraction workspace
  DBuf con_ws, con_desc, con_out;
  DBuf tc_ws, tc_desc, tc_err;
  DBuf oz_ws, oz_desc;
  // the contraction of the unrotated (diagonal) pairs runs on a second stream,
  // beside the rotation kernel, with its own workspace
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mpo = nullptr;
  DBuf oz_ws_side, oz_desc_side, split_out, split_idx;
  DBuf con_ws_side, con_desc_side, bs_flops, bs_flops_side;   // block-sparse FP64 form
  bool no_events = false;                  // profiling events off (work on the side stream)
  bool err_preset = false;                 // the pipeline error word was cleared before the fork
  DBuf solve_buf;                          // tnqe_solve / tnqe_dependence, sized once for M = 32
  // graph capture / replay of whole matrix-element calls
  bool capturing = false;
  std::vector<Upload>* cap_uploads = nullptr;
  std::map<std::vector<long long>, std::unique_ptr<GraphEntry>> graphs;
  std::map<std::vector<long long>, int> seen;   // calls per key: the second identical call captures
  long long generation = 0;                // bumped whenever the set of states changes
  // launch shapes (tnqe_autotune): sliced GEMM N tiles of stages 1 and 3, MPO kernel width (0 = largest that fits)
  struct Tune {
    int oz_bn1 = 128, oz_bn3 = 128, spmm_bw = 0;
    int bs_t1 = 128, bs_t2 = 128, bs_t3 = 128;   // CTA sizes of the charge-block stages
  } tune;
  std::string tune_cache;                   // autotune_cache path ("" = none)
  // last tnqe_rotate result
  int kept_pair_valid = 0;
  std::vector<int> kept_dims;
  std::vector<long long> kept_off;
  double times[3] = {0, 0, 0};
  int launches = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // per-kernel profile of the last matrix-element call (see tnqe_last_profile)
  std::vector<cudaEvent_t> pev;
  double prof[TNQE_PROFILE_LEN] = {};
};

namespace {

tnqe_status fail(tnqe_ctx* c, const Error& e) {
  if (c) c->err = e.what();
  return e.st;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host-to-device copy of planning data.  While a call is being captured the
// copy is recorded for the replays instead (each replay repeats it before the
// graph launch), so the graph itself holds kernels only.
void upload(tnqe_ctx* c, void* dst, const void* src, size_t n) {
  if (n == 0) return;
  if (c->capturing) {
    const unsigned char* b = static_cast<const unsigned char*>(src);
    c->cap_uploads->push_back(Upload{dst, std::vector<unsigned char>(b, b + n)});
    return;
  }
  CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream));
}

// Event on the context stream; while capturing, an event-record node of the graph
// (a plain record inside a capture only orders work and is not replayed).
void record_event(tnqe_ctx* c, cudaEvent_t e) {
  if (c->no_events) return;
  if (c->capturing) CK(cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal));
  else CK(cudaEventRecord(e, c->stream));
}

void clear_graphs(tnqe_ctx* c) {
  c->graphs.clear();
  c->seen.clear();
}

// ----------------------------------------------------------------------------- rotation of a batch
struct RotBatch {
  std::vector<int> pair_idx;             // index into the caller's pair list
  std::vector<int> ii, jj;
  std::vector<std::vector<int>> cap;     // per pair: N + 1 capacities
  std::vector<std::vector<long long>> woff;
  std::vector<long long> work_base;      // doubles, per pair
  std::vector<long long> scratch_base;   // doubles, per pair (theta + wbuf + qbuf)
  std::vector<long long> scratch_len;
  // device views per pair
  std::vector<double*> work;
  std::vector<int*> dims;
  std::vector<SectorTable*> sec;
  std::vector<double*> disc;
  std::vector<int*> status;
  std::vector<double*> flops;
  size_t per_small = 0, o_stat = 0, o_flops = 0;
};

const long long META_INTS = 2 * 32768;

// Givens plans (gates, sites, sides on the device) of every pair (i, j) that has
// none yet, computed on the host and uploaded together: one allocation and one
// copy for the whole batch (an arena freed with the states).
void prepare_plans(tnqe_ctx* c, const std::vector<int>& ii, const std::vector<int>& jj) {
  const int N = c->N;
  struct Host {
    std::pair<int, int> key;
    int ngates, neg_site;
    size_t oG, oS, oD;
  };
  std::vector<Host> todo;
  HostPack pk;
  for (size_t k = 0; k < ii.size(); ++k) {
    const auto key = std::make_pair(ii[k], jj[k]);
    if (c->plans.count(key)) continue;
    bool dup = false;
    for (const Host& h : todo) dup = dup || h.key == key;
    if (dup) continue;
    const std::vector<double>& Ui = c->mps[ii[k]]->U;
    const std::vector<double>& Uj = c->mps[jj[k]]->U;
    std::vector<double> V((size_t)N * N);
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q) {
        double acc = 0.0;
        for (int a = 0; a < N; ++a) acc += Ui[(size_t)a * N + p] * Uj[(size_t)a * N + q];
        V[(size_t)p * N + q] = acc;
      }
    GivensPlan gp = givens_plan(V.data(), N);
    const int ng = (int)gp.gates.size();
    std::vector<double> G((size_t)std::max(1, ng) * 256, 0.0);
    std::vector<int> site(std::max(1, ng)), side(std::max(1, ng));
    for (int g = 0; g < ng; ++g) {
      gate_matrix(gp.gates[g].c, gp.gates[g].s, &G[(size_t)g * 256]);
      site[g] = gp.gates[g].site;
      side[g] = gp.gates[g].side;
    }
    Host h{key, ng, gp.neg_site, pk.add(G), pk.add(site), pk.add(side)};
    todo.push_back(h);
  }
  if (todo.empty()) return;
  void* dev = nullptr;
  CK(cudaMalloc(&dev, pk.h.size()));
  c->plan_arenas.push_back(dev);
  CK(cudaMemcpy(dev, pk.h.data(), pk.h.size(), cudaMemcpyHostToDevice));
  unsigned char* base = static_cast<unsigned char*>(dev);
  for (const Host& h : todo) {
    auto pp = std::make_unique<PairPlan>();
    pp->ngates = h.ngates;
    pp->neg_site = h.neg_site;
    pp->d_gates = reinterpret_cast<double*>(base + h.oG);
    pp->d_site = reinterpret_cast<int*>(base + h.oS);
    pp->d_side = reinterpret_cast<int*>(base + h.oD);
    c->plans.emplace(h.key, std::move(pp));
  }
}

PairPlan* get_plan(tnqe_ctx* c, int i, int j) {
  auto it = c->plans.find(std::make_pair(i, j));
  if (it == c->plans.end()) {
    prepare_plans(c, {i}, {j});
    it = c->plans.find(std::make_pair(i, j));
  }
  return it->second.get();
}

int chi_rot_of(tnqe_ctx* c, int j) { return c->opt.chi_rot > 0 ? c->opt.chi_rot : c->mps[j]->chi; }

// Launch the rotation of every (i, j), i != j, of `pairs`; results stay in rot_work.
void run_rotations(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pairs, RotBatch& rb, int pad_out) {
  const int N = c->N;
  rb = RotBatch{};
  for (size_t p = 0; p < pairs.size(); ++p)
    if (pairs[p].first != pairs[p].second) {
      rb.pair_idx.push_back((int)p);
      rb.ii.push_back(pairs[p].first);
      rb.jj.push_back(pairs[p].second);
    }
  const int np = (int)rb.pair_idx.size();
  if (np == 0) return;
  prepare_plans(c, rb.ii, rb.jj);
  long long work_total = 0, scratch_total = 0;
  for (int k = 0; k < np; ++k) {
    const DevMps& mj = *c->mps[rb.jj[k]];
    const int cr = chi_rot_of(c, rb.jj[k]);
    std::vector<int> cap(N + 1);
    for (int b = 0; b <= N; ++b) cap[b] = std::max(std::min(cr, c->exact_dim[b]), mj.dims[b]);
    if (*std::max_element(cap.begin(), cap.end()) > 256)
      throw Error(TNQE_ERR_ARG, "bond dimension above 256 is not supported by the rotation kernel");
    std::vector<long long> off(N);
    long long tot = 0;
    for (int s = 0; s < N; ++s) {
      off[s] = tot;
      tot += (long long)cap[s] * 4 * cap[s + 1];
    }
    long long th = 16;
    for (int a = 0; a + 1 < N; ++a) th = std::max(th, 16LL * cap[a] * cap[a + 2]);
    for (int a = 0; a < N; ++a) th = std::max(th, 4LL * cap[a] * cap[a + 1]);   // one site at capacity
    rb.cap.push_back(cap);
    rb.woff.push_back(off);
    rb.work_base.push_back(work_total);
    work_total += tot;
    rb.scratch_base.push_back(scratch_total);
    rb.scratch_len.push_back(th);
    scratch_total += 6 * th;
  }
  // small per-pair arrays: dims (N+1 ints), caps, offsets, sectors, disc, status
  auto al256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t sec_bytes = al256(sizeof(SectorTable) * (N + 1));
  const size_t per_small = al256(sec_bytes + 2 * 256 + (size_t)(N + 1) * 8 * 2 + (size_t)N * 8 + 64);
  c->rot_work.ensure(sizeof(double) * std::max<long long>(work_total, 1));
  c->rot_scratch.ensure(sizeof(double) * std::max<long long>(scratch_total, 1));
  c->rot_meta.ensure(sizeof(int) * META_INTS * np);
  c->rot_small.ensure(per_small * np);
  c->rot_desc.ensure(sizeof(RotDesc) * np);
  std::vector<unsigned char> small(per_small * np, 0);
  std::vector<RotDesc> descs(np);
  for (int k = 0; k < np; ++k) {
    unsigned char* hb = small.data() + per_small * k;
    unsigned char* db = c->rot_small.as<unsigned char>() + per_small * k;
    size_t o = 0;
    SectorTable* dsec = reinterpret_cast<SectorTable*>(db + o);
    o += sec_bytes;
    int* ddims = reinterpret_cast<int*>(db + o);
    o += 256;
    int* dcap = reinterpret_cast<int*>(db + o);
    std::memcpy(hb + o, rb.cap[k].data(), sizeof(int) * (N + 1));
    o += 256;
    long long* dwoff = reinterpret_cast<long long*>(db + o);
    std::memcpy(hb + o, rb.woff[k].data(), sizeof(long long) * N);
    o += (size_t)(N + 1) * 8 * 2 + (size_t)N * 8;
    double* ddisc = reinterpret_cast<double*>(db + o);
    double* dflops = reinterpret_cast<double*>(db + o + 8);
    rb.o_flops = o + 8;
    o += 16;
    int* dstat = reinterpret_cast<int*>(db + o);
    rb.o_stat = o;
    const DevMps& mj = *c->mps[rb.jj[k]];
    PairPlan* pl = get_plan(c, rb.ii[k], rb.jj[k]);
    RotDesc& d = descs[k];
    d.N = N;
    d.chi_rot = chi_rot_of(c, rb.jj[k]);
    d.ngates = pl->ngates;
    d.neg_site = pl->neg_site;
    d.renorm = c->opt.renormalize_rotated;
    d.pad_out = pad_out;
    d.max_sweeps = c->opt.max_jacobi_sweeps;
    d.cutoff = c->opt.cutoff;
    d.src = mj.d_t;
    d.src_off = mj.d_off;
    d.src_dims = mj.d_dims;
    d.src_sec = mj.d_sec;
    d.work = c->rot_work.as<double>() + rb.work_base[k];
    d.work_off = dwoff;
    d.work_dims = ddims;
    d.work_cap = dcap;
    d.work_sec = dsec;
    d.gates = pl->d_gates;
    d.gate_site = pl->d_site;
    d.gate_side = pl->d_side;
    double* sb = c->rot_scratch.as<double>() + rb.scratch_base[k];
    const long long th = rb.scratch_len[k];
    d.theta = sb;
    d.bbuf = sb + th;
    d.wbuf = sb + 2 * th;
    d.qbuf = sb + 3 * th;
    d.tbuf = sb + 4 * th;
    d.w32 = reinterpret_cast<float*>(sb + 5 * th);
    d.q32 = d.w32 + th;
    d.meta = c->rot_meta.as<int>() + META_INTS * k;
    d.meta_cap = META_INTS;
    d.discarded = ddisc;
    d.status = dstat;
    d.flops = dflops;
    rb.work.push_back(d.work);
    rb.dims.push_back(ddims);
    rb.sec.push_back(dsec);
    rb.disc.push_back(ddisc);
    rb.status.push_back(dstat);
    rb.flops.push_back(dflops);
  }
  rb.per_small = per_small;
  upload(c, c->rot_small.p, small.data(), small.size());
  // Launch order: the CTAs start in index order and a CTA's time grows with the
  // rotated state's bond dimension, so when the pairs fill more than one wave of
  // SMs the largest rotations go first (each descriptor carries all its pointers;
  // the order changes no result).
  {
    std::vector<int> order(np);
    for (int k = 0; k < np; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return chi_rot_of(c, rb.jj[a]) > chi_rot_of(c, rb.jj[b]); });
    std::vector<RotDesc> launch_descs(np);
    for (int t = 0; t < np; ++t) launch_descs[t] = descs[order[t]];
    descs.swap(launch_descs);
  }
  upload(c, c->rot_desc.p, descs.data(), sizeof(RotDesc) * np);
  record_event(c, c->pev[0]);
  CKL(launch_rotate(c->rot_desc.as<RotDesc>(), np, 0, c->stream));
  c->launches += 1;
  record_event(c, c->pev[1]);
}

// read back dims / discarded / status of a finished rotation batch
void fetch_rotation_results(tnqe_ctx* c, const RotBatch& rb, std::vector<std::vector<int>>& dims,
                            std::vector<double>& disc, int& status_or) {
  const int N = c->N;
  const int np = (int)rb.pair_idx.size();
  dims.assign(np, std::vector<int>(N + 1));
  disc.assign(np, 0.0);
  status_or = 0;
  for (int k = 0; k < np; ++k) {
    CK(cudaMemcpyAsync(dims[k].data(), rb.dims[k], sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&disc[k], rb.disc[k], sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  std::vector<int> st(np);
  std::vector<double> fl(np);
  for (int k = 0; k < np; ++k) {
    CK(cudaMemcpyAsync(&st[k], rb.status[k], sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&fl[k], rb.flops[k], sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < np; ++k) {
    status_or |= st[k];
    c->prof[4] += fl[k];
  }
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->pev[0], c->pev[1]));
  c->prof[0] += ms;
}

// ----------------------------------------------------------------------------- contraction
struct KetView {
  const double* base;
  std::vector<long long> off;   // per site
  std::vector<int> dims;        // N + 1
  const SectorTable* sec = nullptr;   // N + 1 device sector tables (the rotation's for a rotated ket)
};

// Per-site event pairs of the last wave go to the finish step; earlier waves
// (which reuse the workspace) are synchronised and read here.
void site_events(tnqe_ctx* c, FinishInfo& fi, bool last, const std::vector<std::array<int, 3>>& reads) {
  if (last) {
    fi.ev_reads.insert(fi.ev_reads.end(), reads.begin(), reads.end());
    return;
  }
  if (c->capturing) throw Error(TNQE_ERR_STATE, "a captured call must fit one workspace wave");
  fi.single_wave = false;
  CK(cudaStreamSynchronize(c->stream));
  if (c->no_events) return;
  for (const auto& r : reads) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->pev[r[0]], c->pev[r[1]]));
    c->prof[r[2]] += ms;
  }
}

// Bytes of contraction workspace one wave may use: 60 % of the free device
// memory (counting the workspace already held), capped by options.workspace_limit.
double ws_budget(tnqe_ctx* c, size_t avail) {
  const double b = 0.6 * (double)avail;
  return c->opt.workspace_limit > 0 ? std::min(b, (double)c->opt.workspace_limit) : b;
}

void run_contractions(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pairs, const std::vector<KetView>& kets,
                      double* d_H, double* d_S, FinishInfo& fi) {
  const int N = c->N;
  const int np = (int)pairs.size();
  // workspace per pair: two environments, X and Y
  std::vector<long long> envsz(np), xsz(np), ysz(np);
  for (int p = 0; p < np; ++p) {
    const DevMps& bi = *c->mps[pairs[p].first];
    const KetView& kv = kets[p];
    long long e = 1, x = 1, y = 1;
    for (int t = 0; t <= N; ++t) e = std::max(e, (long long)bi.dims[t] * bi.mpo.dims[t] * kv.dims[t]);
    for (int t = 0; t < N; ++t) {
      x = std::max(x, (long long)bi.dims[t] * bi.mpo.dims[t] * 4 * kv.dims[t + 1]);
      y = std::max(y, (long long)bi.dims[t] * 4 * bi.mpo.dims[t + 1] * kv.dims[t + 1]);
    }
    envsz[p] = e;
    xsz[p] = x;
    ysz[p] = y;
  }
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const double budget = ws_budget(c, freeb + c->con_ws.cap);
  // waves of pairs whose workspace fits
  size_t p0 = 0;
  while (p0 < (size_t)np) {
    size_t p1 = p0;
    double need = 0.0;
    while (p1 < (size_t)np) {
      const double add = 8.0 * (2.0 * envsz[p1] + xsz[p1] + ysz[p1]);
      if (p1 > p0 && need + add > budget) break;
      need += add;
      ++p1;
    }
    const int nw = (int)(p1 - p0);
    c->con_ws.ensure((size_t)need + 256);
    std::vector<double*> env0(nw), env1(nw), X(nw), Y(nw);
    {
      double* base = c->con_ws.as<double>();
      long long o = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        env0[w] = base + o;
        o += envsz[p];
        env1[w] = base + o;
        o += envsz[p];
        X[w] = base + o;
        o += xsz[p];
        Y[w] = base + o;
        o += ysz[p];
      }
    }
    // descriptors for all sites of this wave
    std::vector<GemmDesc> g1, g3;
    std::vector<SpmmDesc> sp;
    std::vector<long long> g1pre, g3pre, sppre;
    std::vector<int> g1n, g3n, spn;
    for (int t = 0; t < N; ++t) {
      long long tiles1 = 0, tiles3 = 0, rows = 0;
      int n1 = 0, n3 = 0, ns = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        const int ca = bi.dims[t], ca2 = bi.dims[t + 1];
        const int cb = kv.dims[t], cb2 = kv.dims[t + 1];
        const int Din = bi.mpo.dims[t], Dout = bi.mpo.dims[t + 1];
        double* Lin = (t & 1) ? env1[w] : env0[w];
        double* Lout = (t & 1) ? env0[w] : env1[w];
        GemmDesc d1{};
        d1.M = ca * Din;
        d1.N = 4 * cb2;
        d1.K = cb;
        d1.transA = 0;
        d1.lda = cb;
        d1.ldb = 4 * cb2;
        d1.ldc = 4 * cb2;
        d1.A = Lin;
        d1.B = kv.base + kv.off[t];
        d1.C = X[w];
        g1pre.push_back(tiles1);
        tiles1 += (long long)((d1.M + 63) / 64) * ((d1.N + 63) / 64);
        g1.push_back(d1);
        ++n1;
        SpmmDesc s{};
        s.chi_a = ca;
        s.nrows = 4 * Dout;
        s.ncols_x = 4 * Din;
        s.width = cb2;
        s.rowptr = bi.d_rowptr[t];
        s.col = bi.d_col[t];
        s.val = bi.d_val[t];
        s.X = X[w];
        s.Y = Y[w];
        sppre.push_back(rows);
        rows += (long long)ca * 4 * Dout;
        sp.push_back(s);
        ++ns;
        GemmDesc d3{};
        d3.M = ca2;
        d3.N = Dout * cb2;
        d3.K = 4 * ca;
        d3.transA = 1;
        d3.lda = ca2;
        d3.ldb = Dout * cb2;
        d3.ldc = Dout * cb2;
        d3.A = bi.d_t + bi.off[t];
        d3.B = Y[w];
        d3.C = Lout;
        g3pre.push_back(tiles3);
        tiles3 += (long long)((d3.M + 63) / 64) * ((d3.N + 63) / 64);
        g3.push_back(d3);
        ++n3;
      }
      g1pre.push_back(tiles1);
      g3pre.push_back(tiles3);
      sppre.push_back(rows);
      g1n.push_back(n1);
      g3n.push_back(n3);
      spn.push_back(ns);
    }
    // pack descriptors + prefixes into one upload
    const size_t b1 = g1.size() * sizeof(GemmDesc), b3 = g3.size() * sizeof(GemmDesc), bs = sp.size() * sizeof(SpmmDesc);
    const size_t bp1 = g1pre.size() * 8, bp3 = g3pre.size() * 8, bps = sppre.size() * 8;
    const size_t bf = (size_t)nw * sizeof(double*);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t total = al(b1) + al(b3) + al(bs) + al(bp1) + al(bp3) + al(bps) + al(bf) + al(bf);
    std::vector<unsigned char> host(total, 0);
    size_t o1 = 0, o3 = o1 + al(b1), os = o3 + al(b3), op1 = os + al(bs), op3 = op1 + al(bp1), ops = op3 + al(bp3),
           of = ops + al(bps), oe = of + al(bf);
    std::memcpy(host.data() + oe, env0.data(), bf);
    std::memcpy(host.data() + o1, g1.data(), b1);
    std::memcpy(host.data() + o3, g3.data(), b3);
    std::memcpy(host.data() + os, sp.data(), bs);
    std::memcpy(host.data() + op1, g1pre.data(), bp1);
    std::memcpy(host.data() + op3, g3pre.data(), bp3);
    std::memcpy(host.data() + ops, sppre.data(), bps);
    std::vector<const double*> fin(nw);
    for (int w = 0; w < nw; ++w) fin[w] = (N & 1) ? env1[w] : env0[w];
    std::memcpy(host.data() + of, fin.data(), bf);
    c->con_desc.ensure(total);
    unsigned char* dd = c->con_desc.as<unsigned char>();
    upload(c, dd, host.data(), total);
    CKL(launch_unit_env_f64(reinterpret_cast<double* const*>(dd + oe), nw, c->stream));   // L_0 = 1
    c->launches += 1;
    for (const GemmDesc& d : g1) c->prof[5] += 2.0 * d.M * d.N * d.K;
    for (const GemmDesc& d : g3) c->prof[7] += 2.0 * d.M * d.N * d.K;
    for (int w = 0; w < nw; ++w) {
      const int p = (int)p0 + w;
      const DevMps& bi = *c->mps[pairs[p].first];
      const KetView& kv = kets[p];
      for (int t = 0; t < N; ++t) {
        const double ca = bi.dims[t], cb2 = kv.dims[t + 1];
        c->prof[6] += 8.0 * ca * cb2 * 4.0 * (bi.mpo.dims[t] + bi.mpo.dims[t + 1]);
        c->prof[8] += 2.0 * (double)bi.mpo.sites[t].val.size() * ca * cb2;
      }
    }
    size_t i1 = 0, i3 = 0, is = 0, ip1 = 0, ip3 = 0, ips = 0;
    for (int t = 0; t < N; ++t) {
      const int n1 = g1n[t], n3 = g3n[t], ns = spn[t];
      cudaEvent_t* E = &c->pev[2 + 6 * t];
      record_event(c, E[0]);
      CKL(launch_gemm_f64(reinterpret_cast<GemmDesc*>(dd + o1) + i1, reinterpret_cast<long long*>(dd + op1) + ip1,
                          n1, g1pre[ip1 + n1], c->stream));
      record_event(c, E[1]);
      CKL(launch_spmm_f64(reinterpret_cast<SpmmDesc*>(dd + os) + is, reinterpret_cast<long long*>(dd + ops) + ips,
                          ns, sppre[ips + ns], c->stream));
      record_event(c, E[2]);
      CKL(launch_gemm_f64(reinterpret_cast<GemmDesc*>(dd + o3) + i3, reinterpret_cast<long long*>(dd + op3) + ip3,
                          n3, g3pre[ip3 + n3], c->stream));
      record_event(c, E[3]);
      c->launches += 3;
      i1 += n1;
      i3 += n3;
      is += ns;
      ip1 += n1 + 1;
      ip3 += n3 + 1;
      ips += ns + 1;
    }
    CKL(launch_extract(reinterpret_cast<const double* const*>(dd + of), nw, d_H + p0, d_S + p0, c->stream));
    c->launches += 1;
    std::vector<std::array<int, 3>> reads;
    for (int t = 0; t < N; ++t) {
      const int e = 2 + 6 * t;
      reads.push_back({e, e + 1, 1});
      reads.push_back({e + 1, e + 2, 2});
      reads.push_back({e + 2, e + 3, 3});
    }
    site_events(c, fi, p1 == (size_t)np, reads);
    p0 = p1;
  }
}

// ----------------------------------------------------------------------------- block-sparse FP64 contraction
// The dense form's workspace and layout, with only the charge-allowed blocks
// computed (kernels_block.cu).  Work items per site: stage 1 and stage 3 one
// CTA per (pair, bra sector, channel class), stage 2 one CTA per (pair, bra
// index).  Algorithmic FLOPs are counted on the device (the ket's sector
// dimensions are decided there) and read back when the call has finished.
// Profiling events of site t of workspace wave w: wave 0 uses the context's
// per-site slots, later waves slots appended after the slicing events.
int wave_event(tnqe_ctx* c, int w, int t) {
  const int N = c->N;
  const int idx = w == 0 ? 2 + 6 * t : 4 + 6 * N * w + 6 * t;
  while ((int)c->pev.size() < idx + 6) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreate(&e));
    c->pev.push_back(e);
  }
  return idx;
}

void run_contractions_bs(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pairs, const std::vector<KetView>& kets,
                         double* d_H, double* d_S, FinishInfo& fi) {
  const int N = c->N;
  const int np = (int)pairs.size();
  std::vector<long long> envsz(np), xsz(np), ysz(np);
  for (int p = 0; p < np; ++p) {
    const DevMps& bi = *c->mps[pairs[p].first];
    const KetView& kv = kets[p];
    long long e = 1, x = 1, y = 1;
    for (int t = 0; t <= N; ++t) e = std::max(e, (long long)bi.dims[t] * bi.mpo.dims[t] * kv.dims[t]);
    for (int t = 0; t < N; ++t) {
      x = std::max(x, (long long)bi.dims[t] * bi.mpo.dims[t] * 4 * kv.dims[t + 1]);
      y = std::max(y, (long long)bi.dims[t] * 4 * bi.mpo.dims[t + 1] * kv.dims[t + 1]);
    }
    envsz[p] = e;
    xsz[p] = x;
    ysz[p] = y;
  }
  c->bs_flops.ensure(4 * sizeof(double));
  CK(cudaMemsetAsync(c->bs_flops.p, 0, 4 * sizeof(double), c->stream));
  double* dfl = c->bs_flops.as<double>();
  fi.bs_flops.push_back(dfl);
  // waves of pairs whose workspace fits in 60 % of the free memory; the waves
  // reuse the workspace in stream order, so no host synchronisation is needed
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const double budget = ws_budget(c, freeb + c->con_ws.cap);
  std::vector<std::pair<int, int>> waves;
  double need_max = 0.0;
  for (int p0 = 0; p0 < np;) {
    int p1 = p0;
    double need = 0.0;
    while (p1 < np) {
      const double add = 8.0 * (2.0 * envsz[p1] + xsz[p1] + ysz[p1]);
      if (p1 > p0 && need + add > budget) break;
      need += add;
      ++p1;
    }
    waves.push_back({p0, p1});
    need_max = std::max(need_max, need);
    p0 = p1;
  }
  c->con_ws.ensure((size_t)need_max + 256);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  struct WaveLayout {
    size_t base, od, op1, op2, op3, oe, of;
    int nw;
    std::vector<long long> tot1, tot2, tot3;
  };
  std::vector<WaveLayout> lay(waves.size());
  std::vector<unsigned char> host;
  for (size_t wv = 0; wv < waves.size(); ++wv) {
    const int p0 = waves[wv].first, nw = waves[wv].second - waves[wv].first;
    std::vector<double*> env0(nw), env1(nw), X(nw), Y(nw);
    {
      double* base = c->con_ws.as<double>();
      long long o = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = p0 + w;
        env0[w] = base + o;
        o += envsz[p];
        env1[w] = base + o;
        o += envsz[p];
        X[w] = base + o;
        o += xsz[p];
        Y[w] = base + o;
        o += ysz[p];
      }
    }
    // descriptors: site-major, pairs inside; CTA prefixes per site and stage
    std::vector<BsSiteDesc> ds((size_t)N * nw);
    std::vector<long long> pre1, pre2, pre3;
    WaveLayout& L = lay[wv];
    L.nw = nw;
    L.tot1.resize(N);
    L.tot2.resize(N);
    L.tot3.resize(N);
    for (int t = 0; t < N; ++t) {
      long long n1 = 0, n2 = 0, n3 = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        BsSiteDesc& d = ds[(size_t)t * nw + w];
        d.Din = bi.mpo.dims[t];
        d.Dout = bi.mpo.dims[t + 1];
        d.ca = bi.dims[t];
        d.ca2 = bi.dims[t + 1];
        d.capb = kv.dims[t];
        d.capb2 = kv.dims[t + 1];
        d.A = bi.d_t + bi.off[t];
        d.B = kv.base + kv.off[t];
        d.braL = bi.d_sec + t;
        d.braR = bi.d_sec + t + 1;
        d.ketL = kv.sec + t;
        d.ketR = kv.sec + t + 1;
        d.Lin = (t & 1) ? env1[w] : env0[w];
        d.Lout = (t & 1) ? env0[w] : env1[w];
        d.X = X[w];
        d.Y = Y[w];
        d.rowptr = bi.d_rowptr[t];
        d.col = bi.d_col[t];
        d.val = bi.d_val[t];
        d.chL = bi.bs_ch[t];
        d.chR = bi.bs_ch[t + 1];
        d.rows = bi.bs_rows[t];
        pre1.push_back(n1);
        pre2.push_back(n2);
        pre3.push_back(n3);
        n1 += (long long)bi.sec[t].nsec * d.chL.ncls;
        n2 += d.ca;
        n3 += (long long)bi.sec[t + 1].nsec * d.chR.ncls;
      }
      pre1.push_back(n1);
      pre2.push_back(n2);
      pre3.push_back(n3);
      L.tot1[t] = n1;
      L.tot2[t] = n2;
      L.tot3[t] = n3;
    }
    const size_t bd = ds.size() * sizeof(BsSiteDesc), bp = pre1.size() * 8, bf = (size_t)nw * sizeof(double*);
    L.base = al(host.size());
    L.od = 0;
    L.op1 = al(bd);
    L.op2 = L.op1 + al(bp);
    L.op3 = L.op2 + al(bp);
    L.oe = L.op3 + al(bp);
    L.of = L.oe + al(bf);
    host.resize(L.base + L.of + al(bf), 0);
    unsigned char* h = host.data() + L.base;
    std::memcpy(h + L.od, ds.data(), bd);
    std::memcpy(h + L.op1, pre1.data(), bp);
    std::memcpy(h + L.op2, pre2.data(), bp);
    std::memcpy(h + L.op3, pre3.data(), bp);
    std::memcpy(h + L.oe, env0.data(), bf);
    std::vector<const double*> fin(nw);
    for (int w = 0; w < nw; ++w) fin[w] = (N & 1) ? env1[w] : env0[w];
    std::memcpy(h + L.of, fin.data(), bf);
  }
  for (size_t wv = 0; wv < waves.size(); ++wv) wave_event(c, (int)wv, N - 1);   // events exist before any launch
  c->con_desc.ensure(host.size());
  upload(c, c->con_desc.p, host.data(), host.size());
  std::vector<std::array<int, 3>> reads;
  for (size_t wv = 0; wv < waves.size(); ++wv) {
    const WaveLayout& L = lay[wv];
    const int nw = L.nw, p0 = waves[wv].first;
    unsigned char* dd = c->con_desc.as<unsigned char>() + L.base;
    CKL(launch_unit_env_f64(reinterpret_cast<double* const*>(dd + L.oe), nw, c->stream));   // L_0 = 1
    c->launches += 1;
    const BsSiteDesc* dsd = reinterpret_cast<const BsSiteDesc*>(dd + L.od);
    for (int t = 0; t < N; ++t) {
      const size_t pofs = (size_t)t * (nw + 1);
      const int e = wave_event(c, (int)wv, t);
      cudaEvent_t* E = &c->pev[e];
      record_event(c, E[0]);
      CKL(launch_bs_stage1(dsd + (size_t)t * nw, reinterpret_cast<const long long*>(dd + L.op1) + pofs, nw,
                           L.tot1[t], dfl, c->tune.bs_t1, c->stream));
      record_event(c, E[1]);
      CKL(launch_bs_stage2(dsd + (size_t)t * nw, reinterpret_cast<const long long*>(dd + L.op2) + pofs, nw,
                           L.tot2[t], dfl, c->tune.bs_t2, c->stream));
      record_event(c, E[2]);
      CKL(launch_bs_stage3(dsd + (size_t)t * nw, reinterpret_cast<const long long*>(dd + L.op3) + pofs, nw,
                           L.tot3[t], dfl, c->tune.bs_t3, c->stream));
      record_event(c, E[3]);
      c->launches += 3;
      reads.push_back({e, e + 1, 1});
      reads.push_back({e + 1, e + 2, 2});
      reads.push_back({e + 2, e + 3, 3});
    }
    CKL(launch_extract(reinterpret_cast<const double* const*>(dd + L.of), nw, d_H + p0, d_S + p0, c->stream));
    c->launches += 1;
  }
  if (!c->no_events) fi.ev_reads.insert(fi.ev_reads.end(), reads.begin(), reads.end());
  fi.waves = std::max(fi.waves, (int)waves.size());
}

// ----------------------------------------------------------------------------- split-precision contraction
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error(TNQE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D FP32 tensor map: rows x cols (cols contiguous, row stride ld floats), 32-column boxes
void encode_map(CUtensorMap* map, const float* base, long long rows, long long cols, long long ld, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = tensor_map_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(TNQE_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

inline long long al64(long long x) { return (x + 63) & ~63LL; }   // floats -> 256-byte aligned offsets
inline int ld4(int x) { return (x + 3) & ~3; }

void run_contractions_tc(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pairs, const std::vector<KetView>& kets,
                         double* d_H, double* d_S, FinishInfo& fi) {
  const int N = c->N;
  const int np = (int)pairs.size();
  // per-pair FP32 workspace: two environments, X, Yt, packed ket / bra sites
  std::vector<long long> envsz(np), xsz(np), ysz(np), packsz(np);
  for (int p = 0; p < np; ++p) {
    const DevMps& bi = *c->mps[pairs[p].first];
    const KetView& kv = kets[p];
    long long e = 4, x = 4, y = 4, pk = 0;
    for (int t = 0; t <= N; ++t) e = std::max(e, (long long)bi.dims[t] * bi.mpo.dims[t] * ld4(kv.dims[t]));
    for (int t = 0; t < N; ++t) {
      x = std::max(x, (long long)bi.dims[t] * bi.mpo.dims[t] * 4 * kv.dims[t + 1]);
      y = std::max(y, (long long)bi.mpo.dims[t + 1] * kv.dims[t + 1] * 4 * bi.dims[t]);
      pk += al64((long long)4 * kv.dims[t + 1] * ld4(kv.dims[t])) + al64((long long)bi.dims[t + 1] * 4 * bi.dims[t]);
    }
    envsz[p] = al64(e);
    xsz[p] = al64(x);
    ysz[p] = al64(y);
    packsz[p] = pk;
  }
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const double budget = ws_budget(c, freeb + c->tc_ws.cap);
  c->tc_err.ensure(256);
  if (!c->err_preset) CK(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
  size_t p0 = 0;
  while (p0 < (size_t)np) {
    size_t p1 = p0;
    double need = 0.0;
    while (p1 < (size_t)np) {
      const double add = 4.0 * (2.0 * envsz[p1] + xsz[p1] + ysz[p1] + packsz[p1]);
      if (p1 > p0 && need + add > budget) break;
      need += add;
      ++p1;
    }
    const int nw = (int)(p1 - p0);
    c->tc_ws.ensure((size_t)need + 1024);
    float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(c->tc_ws.p) + 255) & ~(uintptr_t)255);
    std::vector<float*> env0(nw), env1(nw), X(nw), Y(nw);
    std::vector<std::vector<float*>> ketT(nw, std::vector<float*>(N)), braT(nw, std::vector<float*>(N));
    std::vector<PackDesc> packs;
    std::vector<long long> packpre;
    long long packtot = 0;
    {
      long long o = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        env0[w] = base + o; o += envsz[p];
        env1[w] = base + o; o += envsz[p];
        X[w] = base + o; o += xsz[p];
        Y[w] = base + o; o += ysz[p];
        for (int t = 0; t < N; ++t) {
          ketT[w][t] = base + o;
          o += al64((long long)4 * kv.dims[t + 1] * ld4(kv.dims[t]));
          braT[w][t] = base + o;
          o += al64((long long)bi.dims[t + 1] * 4 * bi.dims[t]);
          PackDesc pk{kv.base + kv.off[t], ketT[w][t], kv.dims[t], kv.dims[t + 1], ld4(kv.dims[t]), 0};
          packpre.push_back(packtot);
          packtot += (long long)kv.dims[t] * 4 * kv.dims[t + 1];
          packs.push_back(pk);
          PackDesc pb{bi.d_t + bi.off[t], braT[w][t], bi.dims[t], bi.dims[t + 1], 4 * bi.dims[t], 1};
          packpre.push_back(packtot);
          packtot += (long long)bi.dims[t] * 4 * bi.dims[t + 1];
          packs.push_back(pb);
        }
      }
    }
    // GEMM / MPO descriptors of every site of this wave
    std::vector<TcGemmDesc> g1, g3;
    std::vector<SpmmTDesc> sp;
    std::vector<long long> g1pre, g3pre, sppre;
    std::vector<int> g1n, g3n, spn;
    for (int t = 0; t < N; ++t) {
      long long tiles1 = 0, tiles3 = 0, tasks = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        const int ca = bi.dims[t], ca2 = bi.dims[t + 1];
        const int cb = kv.dims[t], cb2 = kv.dims[t + 1];
        const int Din = bi.mpo.dims[t], Dout = bi.mpo.dims[t + 1];
        float* Lin = (t & 1) ? env1[w] : env0[w];
        float* Lout = (t & 1) ? env0[w] : env1[w];
        TcGemmDesc d1;
        std::memset(&d1, 0, sizeof(d1));
        d1.M = ca * Din;
        d1.N = 4 * cb2;
        d1.K = cb;
        encode_map(&d1.mapA, Lin, d1.M, cb, ld4(cb), TC_BM);
        encode_map(&d1.mapB, ketT[w][t], d1.N, cb, ld4(cb), TC_BN);
        d1.C = X[w];
        d1.ldc = d1.N;
        d1.cg = d1.N;
        d1.cld = 0;
        d1.tiles_n = (d1.N + TC_BN - 1) / TC_BN;
        g1pre.push_back(tiles1);
        tiles1 += (long long)((d1.M + TC_BM - 1) / TC_BM) * d1.tiles_n;
        g1.push_back(d1);
        SpmmTDesc s{};
        s.rowptr = bi.d_rowptr[t];
        s.col = bi.d_col[t];
        s.val = bi.d_val32[t];
        s.X = X[w];
        s.Yt = Y[w];
        s.chi_a = ca;
        s.Din = Din;
        s.Dout = Dout;
        s.width = cb2;
        s.ldy = 4 * ca;
        sppre.push_back(tasks);
        tasks += (long long)Dout * ((cb2 + 31) / 32) * ((ca + 31) / 32);
        sp.push_back(s);
        TcGemmDesc d3;
        std::memset(&d3, 0, sizeof(d3));
        d3.M = ca2;
        d3.N = Dout * cb2;
        d3.K = 4 * ca;
        encode_map(&d3.mapA, braT[w][t], ca2, d3.K, d3.K, TC_BM);
        encode_map(&d3.mapB, Y[w], d3.N, d3.K, d3.K, TC_BN);
        d3.C = Lout;
        d3.ldc = (long long)Dout * ld4(cb2);
        d3.cg = cb2;
        d3.cld = ld4(cb2);
        d3.tiles_n = (d3.N + TC_BN - 1) / TC_BN;
        g3pre.push_back(tiles3);
        tiles3 += (long long)((d3.M + TC_BM - 1) / TC_BM) * d3.tiles_n;
        g3.push_back(d3);
      }
      g1pre.push_back(tiles1);
      g3pre.push_back(tiles3);
      sppre.push_back(tasks);
      g1n.push_back(nw);
      g3n.push_back(nw);
      spn.push_back(nw);
    }
    for (const TcGemmDesc& d : g1) c->prof[5] += 2.0 * d.M * d.N * d.K;
    for (const TcGemmDesc& d : g3) c->prof[7] += 2.0 * d.M * d.N * d.K;
    for (int w = 0; w < nw; ++w) {
      const int p = (int)p0 + w;
      const DevMps& bi = *c->mps[pairs[p].first];
      const KetView& kv = kets[p];
      for (int t = 0; t < N; ++t) {
        const double ca = bi.dims[t], cb2 = kv.dims[t + 1];
        c->prof[6] += 4.0 * ca * cb2 * 4.0 * (bi.mpo.dims[t] + bi.mpo.dims[t + 1]);
        c->prof[8] += 2.0 * (double)bi.mpo.sites[t].val.size() * ca * cb2;
      }
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b1 = g1.size() * sizeof(TcGemmDesc), b3 = g3.size() * sizeof(TcGemmDesc);
    const size_t bs = sp.size() * sizeof(SpmmTDesc), bpk = packs.size() * sizeof(PackDesc);
    const size_t bp1 = g1pre.size() * 8, bp3 = g3pre.size() * 8, bps = sppre.size() * 8, bpp = (packpre.size() + 1) * 8;
    const size_t bf = (size_t)nw * sizeof(float*);
    const size_t o1 = 0, o3 = o1 + al(b1), os = o3 + al(b3), opk = os + al(bs), op1 = opk + al(bpk),
                 op3 = op1 + al(bp1), ops = op3 + al(bp3), opp = ops + al(bps), of = opp + al(bpp), oe = of + al(bf);
    const size_t total = oe + al(bf);
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + oe, env0.data(), bf);
    std::memcpy(host.data() + o1, g1.data(), b1);
    std::memcpy(host.data() + o3, g3.data(), b3);
    std::memcpy(host.data() + os, sp.data(), bs);
    std::memcpy(host.data() + opk, packs.data(), bpk);
    std::memcpy(host.data() + op1, g1pre.data(), bp1);
    std::memcpy(host.data() + op3, g3pre.data(), bp3);
    std::memcpy(host.data() + ops, sppre.data(), bps);
    packpre.push_back(packtot);
    std::memcpy(host.data() + opp, packpre.data(), bpp);
    std::vector<const float*> fin(nw);
    for (int w = 0; w < nw; ++w) fin[w] = (N & 1) ? env1[w] : env0[w];
    std::memcpy(host.data() + of, fin.data(), bf);
    c->tc_desc.ensure(total);
    unsigned char* dd = c->tc_desc.as<unsigned char>();
    upload(c, dd, host.data(), total);
    CKL(launch_unit_env_f32(reinterpret_cast<float* const*>(dd + oe), nw, c->stream));   // L_0 = 1
    c->launches += 1;
    CKL(launch_pack_sites(reinterpret_cast<PackDesc*>(dd + opk), reinterpret_cast<long long*>(dd + opp),
                          (int)packs.size(), packtot, c->stream));
    c->launches += 1;
    int* derr = c->tc_err.as<int>();
    size_t i1 = 0, i3 = 0, is = 0, ip1 = 0, ip3 = 0, ips = 0;
    for (int t = 0; t < N; ++t) {
      const int n1 = g1n[t], n3 = g3n[t], ns = spn[t];
      cudaEvent_t* E = &c->pev[2 + 6 * t];
      record_event(c, E[0]);
      CKL(launch_gemm_tf32x3(reinterpret_cast<TcGemmDesc*>(dd + o1) + i1, reinterpret_cast<long long*>(dd + op1) + ip1,
                             n1, g1pre[ip1 + n1], c->opt.max_spin, derr, c->stream));
      record_event(c, E[1]);
      CKL(launch_spmm_t_f32(reinterpret_cast<SpmmTDesc*>(dd + os) + is, reinterpret_cast<long long*>(dd + ops) + ips,
                            ns, sppre[ips + ns], c->stream));
      record_event(c, E[2]);
      CKL(launch_gemm_tf32x3(reinterpret_cast<TcGemmDesc*>(dd + o3) + i3, reinterpret_cast<long long*>(dd + op3) + ip3,
                             n3, g3pre[ip3 + n3], c->opt.max_spin, derr, c->stream));
      record_event(c, E[3]);
      c->launches += 3;
      i1 += n1;
      i3 += n3;
      is += ns;
      ip1 += n1 + 1;
      ip3 += n3 + 1;
      ips += ns + 1;
    }
    CKL(launch_extract_f32(reinterpret_cast<const float* const*>(dd + of), nw, 4, d_H + p0, d_S + p0, c->stream));
    c->launches += 1;
    std::vector<std::array<int, 3>> reads;
    for (int t = 0; t < N; ++t) {
      const int e = 2 + 6 * t;
      reads.push_back({e, e + 1, 1});
      reads.push_back({e + 1, e + 2, 2});
      reads.push_back({e + 2, e + 3, 3});
    }
    site_events(c, fi, p1 == (size_t)np, reads);
    p0 = p1;
  }
  fi.check_err = true;
}


// ----------------------------------------------------------------------------- sliced-BF16 contraction
inline long long ld8(long long x) { return (x + 7) & ~7LL; }
inline size_t lz8(size_t x) { return (x + 7) & ~(size_t)7; }
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// 3-D BF16 tensor map over slices [ns][rows][ldK] (K contiguous), box {32, box_rows, ns}, 64-byte swizzle
void encode_slices(CUtensorMap* map, const __nv_bfloat16* base, long long rows, long long K, long long ldK, int ns,
                   int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)ns};
  cuuint64_t strides[2] = {(cuuint64_t)ldK * 2, (cuuint64_t)rows * ldK * 2};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)ns};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = tensor_map_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                          const_cast<__nv_bfloat16*>(base), dims, strides, box, es,
                                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(TNQE_ERR_CUDA, "cuTensorMapEncodeTiled (slices) failed: " + std::to_string((int)r));
}

int slices_of(int precision) {
  return precision == TNQE_PREC_BF16X3 ? 2 : precision == TNQE_PREC_BF16X6 ? 3 : precision == TNQE_PREC_BF16X10 ? 4 : 5;
}

void run_contractions_oz(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pairs, const std::vector<KetView>& kets,
                         double* d_H, double* d_S, FinishInfo& fi) {
  const int N = c->N;
  const int np = (int)pairs.size();
  const int ns = slices_of(c->opt.precision);
  // per-pair workspace (bytes): environment, X / B-slices, Y / A-slices, exponents, site slices
  std::vector<size_t> envb(np), xbb(np), yab(np), expb(np), siteb(np);
  for (int p = 0; p < np; ++p) {
    const DevMps& bi = *c->mps[pairs[p].first];
    const KetView& kv = kets[p];
    size_t e = 8, xb = 8, ya = 8, ex = 4, st = 0;
    for (int t = 0; t <= N; ++t) e = std::max(e, (size_t)bi.dims[t] * bi.mpo.dims[t] * kv.dims[t] * 8);
    for (int t = 0; t < N; ++t) {
      const size_t ca = bi.dims[t], ca2 = bi.dims[t + 1], cb = kv.dims[t], cb2 = kv.dims[t + 1];
      const size_t Din = bi.mpo.dims[t], Dout = bi.mpo.dims[t + 1];
      if (4 * ca > (size_t)OZ_MAXK || cb > (size_t)OZ_MAXK)
        throw Error(TNQE_ERR_ARG, "sliced BF16 contraction needs bond dimensions <= 256");
      xb = std::max(xb, std::max(ca * Din * 4 * cb2 * 8, (size_t)ns * Dout * cb2 * lz8(4 * ca) * 2));
      ya = std::max(ya, std::max(ca * 4 * Dout * cb2 * 8, (size_t)ns * ca * Din * lz8(cb) * 2));
      ex = std::max(ex, std::max(ca * Din, Dout * cb2) * 4);
      st += al256((size_t)ns * 4 * cb2 * lz8(cb) * 2) + al256(4 * cb2 * 4) + al256((size_t)ns * ca2 * lz8(4 * ca) * 2) +
            al256(ca2 * 4);
    }
    envb[p] = al256(e);
    xbb[p] = al256(xb);
    yab[p] = al256(ya);
    expb[p] = 2 * al256(ex);
    siteb[p] = st;
  }
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const double budget = ws_budget(c, freeb + c->oz_ws.cap);
  c->tc_err.ensure(256);
  if (!c->err_preset) CK(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
  int* derr = c->tc_err.as<int>();
  size_t p0 = 0;
  while (p0 < (size_t)np) {
    size_t p1 = p0;
    double need = 0.0;
    while (p1 < (size_t)np) {
      const double add = (double)(envb[p1] + xbb[p1] + yab[p1] + expb[p1] + siteb[p1]);
      if (p1 > p0 && need + add > budget) break;
      need += add;
      ++p1;
    }
    const int nw = (int)(p1 - p0);
    c->oz_ws.ensure((size_t)need + 1024);
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(c->oz_ws.p) + 255) & ~(uintptr_t)255);
    std::vector<float2*> env(nw), X(nw), Y(nw);
    std::vector<__nv_bfloat16*> Bsl(nw), Asl(nw);
    std::vector<int*> expA(nw), expB(nw);
    std::vector<std::vector<__nv_bfloat16*>> ketS(nw, std::vector<__nv_bfloat16*>(N)), braS(nw, std::vector<__nv_bfloat16*>(N));
    std::vector<std::vector<int*>> ketE(nw, std::vector<int*>(N)), braE(nw, std::vector<int*>(N));
    std::vector<SliceSiteDesc> sites;
    std::vector<long long> sitepre;
    long long siterows = 0;
    {
      size_t o = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        env[w] = reinterpret_cast<float2*>(base + o); o += envb[p];
        X[w] = reinterpret_cast<float2*>(base + o);
        Bsl[w] = reinterpret_cast<__nv_bfloat16*>(base + o); o += xbb[p];
        Y[w] = reinterpret_cast<float2*>(base + o);
        Asl[w] = reinterpret_cast<__nv_bfloat16*>(base + o); o += yab[p];
        expA[w] = reinterpret_cast<int*>(base + o); o += expb[p] / 2;
        expB[w] = reinterpret_cast<int*>(base + o); o += expb[p] / 2;
        for (int t = 0; t < N; ++t) {
          const int ca = bi.dims[t], ca2 = bi.dims[t + 1], cb = kv.dims[t], cb2 = kv.dims[t + 1];
          ketS[w][t] = reinterpret_cast<__nv_bfloat16*>(base + o); o += al256((size_t)ns * 4 * cb2 * lz8(cb) * 2);
          ketE[w][t] = reinterpret_cast<int*>(base + o); o += al256((size_t)4 * cb2 * 4);
          braS[w][t] = reinterpret_cast<__nv_bfloat16*>(base + o); o += al256((size_t)ns * ca2 * lz8(4 * ca) * 2);
          braE[w][t] = reinterpret_cast<int*>(base + o); o += al256((size_t)ca2 * 4);
          SliceSiteDesc k{kv.base + kv.off[t], ketS[w][t], ketE[w][t], ld8(cb), (long long)4 * cb2 * ld8(cb), cb, cb2, 0, ns};
          sitepre.push_back(siterows);
          siterows += 4LL * cb2;
          sites.push_back(k);
          SliceSiteDesc b{bi.d_t + bi.off[t], braS[w][t], braE[w][t], ld8(4 * ca), (long long)ca2 * ld8(4 * ca), ca, ca2,
                          1, ns};
          sitepre.push_back(siterows);
          siterows += ca2;
          sites.push_back(b);
        }
      }
    }
    int max_ncx = 4;
    for (int w = 0; w < nw; ++w)
      for (int t = 0; t < N; ++t) max_ncx = std::max(max_ncx, 4 * c->mps[pairs[p0 + w].first]->mpo.dims[t]);
    int spmm_bw = spmm_df_smem_width(max_ncx);
    if (c->tune.spmm_bw > 0 && spmm_bw > 0) spmm_bw = std::min(spmm_bw, c->tune.spmm_bw);
    const int bn1 = c->tune.oz_bn1, bn3 = c->tune.oz_bn3;
    std::vector<SliceRowsDesc> sa;
    std::vector<SliceColsDesc> sb;
    std::vector<OzGemmDesc> g1, g3;
    std::vector<SpmmDfDesc> sp;
    std::vector<long long> sapre, sbpre, g1pre, g3pre, sppre;
    std::vector<int> sbmaxk(N, 0);        // largest K of the column slicing per site
    double slice_bytes = 0.0;
    for (int t = 0; t < N; ++t) {
      long long rowsA = 0, blocksB = 0, tiles1 = 0, tiles3 = 0, tasks = 0;
      for (int w = 0; w < nw; ++w) {
        const int p = (int)p0 + w;
        const DevMps& bi = *c->mps[pairs[p].first];
        const KetView& kv = kets[p];
        const int ca = bi.dims[t], ca2 = bi.dims[t + 1], cb = kv.dims[t], cb2 = kv.dims[t + 1];
        const int Din = bi.mpo.dims[t], Dout = bi.mpo.dims[t + 1];
        const long long MA = (long long)ca * Din;
        // A slices: environment rows (a, w) over b
        SliceRowsDesc a{env[w], Asl[w], expA[w], cb, ld8(cb), MA * ld8(cb), cb, ns};
        sapre.push_back(rowsA);
        rowsA += MA;
        sa.push_back(a);
        slice_bytes += (double)MA * cb * (8.0 + 2.0 * ns);
        OzGemmDesc d1;
        std::memset(&d1, 0, sizeof(d1));
        d1.M = (int)MA;
        d1.N = 4 * cb2;
        d1.K = cb;
        encode_slices(&d1.mapA, Asl[w], MA, cb, ld8(cb), ns, OZ_BM);
        encode_slices(&d1.mapB, ketS[w][t], 4LL * cb2, cb, ld8(cb), ns, bn1);
        d1.ea = expA[w];
        d1.eb = ketE[w][t];
        d1.C = X[w];
        d1.ldc = d1.N;
        d1.tiles_n = (d1.N + bn1 - 1) / bn1;
        d1.nslices = ns;
        g1pre.push_back(tiles1);
        tiles1 += (long long)((d1.M + OZ_BM - 1) / OZ_BM) * d1.tiles_n;
        g1.push_back(d1);
        SpmmDfDesc s{};
        s.chi_a = ca;
        s.nrows = 4 * Dout;
        s.ncols_x = 4 * Din;
        s.width = cb2;
        s.rowptr = bi.d_rowptr[t];
        s.rowperm = bi.d_rowperm[t];
        s.col = bi.d_col[t];
        s.val = bi.d_valdf[t];
        s.ent = bi.d_ent[t];
        s.X = X[w];
        s.Y = Y[w];
        sppre.push_back(tasks);
        tasks += spmm_bw ? (long long)ca * ((cb2 + spmm_bw - 1) / spmm_bw) : (long long)ca * 4 * Dout;
        sp.push_back(s);
        // B slices: Y columns (w', b') over (a, k), K-major
        const long long NB = (long long)Dout * cb2;
        SliceColsDesc b{Y[w], Bsl[w], expB[w], NB, ld8(4 * ca), NB * ld8(4 * ca), 4 * ca, (int)NB, ns, 0};
        sbmaxk[t] = std::max(sbmaxk[t], 4 * ca);
        sbpre.push_back(blocksB);
        blocksB += (NB + 15) / 16;
        sb.push_back(b);
        slice_bytes += (double)NB * 4 * ca * (8.0 + 2.0 * ns);
        OzGemmDesc d3;
        std::memset(&d3, 0, sizeof(d3));
        d3.M = ca2;
        d3.N = (int)NB;
        d3.K = 4 * ca;
        encode_slices(&d3.mapA, braS[w][t], ca2, 4LL * ca, ld8(4 * ca), ns, OZ_BM);
        encode_slices(&d3.mapB, Bsl[w], NB, 4LL * ca, ld8(4 * ca), ns, bn3);
        d3.ea = braE[w][t];
        d3.eb = expB[w];
        d3.C = env[w];
        d3.ldc = NB;
        d3.tiles_n = (d3.N + bn3 - 1) / bn3;
        d3.nslices = ns;
        g3pre.push_back(tiles3);
        tiles3 += (long long)((d3.M + OZ_BM - 1) / OZ_BM) * d3.tiles_n;
        g3.push_back(d3);
      }
      sapre.push_back(rowsA);
      sbpre.push_back(blocksB);
      g1pre.push_back(tiles1);
      g3pre.push_back(tiles3);
      sppre.push_back(tasks);
    }
    for (const OzGemmDesc& d : g1) c->prof[5] += 2.0 * d.M * d.N * d.K;
    for (const OzGemmDesc& d : g3) c->prof[7] += 2.0 * d.M * d.N * d.K;
    c->prof[11] += slice_bytes;
    for (int w = 0; w < nw; ++w) {
      const int p = (int)p0 + w;
      const DevMps& bi = *c->mps[pairs[p].first];
      const KetView& kv = kets[p];
      for (int t = 0; t < N; ++t) {
        const double ca = bi.dims[t], cb2 = kv.dims[t + 1];
        c->prof[6] += 8.0 * ca * cb2 * 4.0 * (bi.mpo.dims[t] + bi.mpo.dims[t + 1]);
        c->prof[8] += 2.0 * (double)bi.mpo.sites[t].val.size() * ca * cb2;
      }
    }
    // one upload: descriptors, prefixes, environment pointers
    sitepre.push_back(siterows);
    struct Blob {
      std::vector<unsigned char> h;
      size_t put(const void* src, size_t n) {
        const size_t o = al256(h.size());
        h.resize(o + al256(n), 0);
        if (n) std::memcpy(h.data() + o, src, n);
        return o;
      }
    } blob;
    const size_t o_g1 = blob.put(g1.data(), g1.size() * sizeof(OzGemmDesc));
    const size_t o_g3 = blob.put(g3.data(), g3.size() * sizeof(OzGemmDesc));
    const size_t o_sa = blob.put(sa.data(), sa.size() * sizeof(SliceRowsDesc));
    const size_t o_sb = blob.put(sb.data(), sb.size() * sizeof(SliceColsDesc));
    const size_t o_sp = blob.put(sp.data(), sp.size() * sizeof(SpmmDfDesc));
    const size_t o_st = blob.put(sites.data(), sites.size() * sizeof(SliceSiteDesc));
    const size_t o_g1p = blob.put(g1pre.data(), g1pre.size() * 8);
    const size_t o_g3p = blob.put(g3pre.data(), g3pre.size() * 8);
    const size_t o_sap = blob.put(sapre.data(), sapre.size() * 8);
    const size_t o_sbp = blob.put(sbpre.data(), sbpre.size() * 8);
    const size_t o_spp = blob.put(sppre.data(), sppre.size() * 8);
    const size_t o_stp = blob.put(sitepre.data(), sitepre.size() * 8);
    const size_t o_env = blob.put(env.data(), env.size() * sizeof(float2*));
    c->oz_desc.ensure(blob.h.size());
    unsigned char* dd = c->oz_desc.as<unsigned char>();
    upload(c, dd, blob.h.data(), blob.h.size());
    record_event(c, c->pev[2 + 6 * N]);
    CKL(launch_unit_env(reinterpret_cast<float2* const*>(dd + o_env), nw, c->stream));
    CKL(launch_slice_sites(reinterpret_cast<SliceSiteDesc*>(dd + o_st), reinterpret_cast<long long*>(dd + o_stp),
                           (int)sites.size(), siterows, c->stream));
    record_event(c, c->pev[3 + 6 * N]);
    c->launches += 2;
    size_t i = 0, ip = 0;
    for (int t = 0; t < N; ++t, i += nw, ip += nw + 1) {
      cudaEvent_t* E = &c->pev[2 + 6 * t];
      auto pre = [&](size_t off) { return reinterpret_cast<long long*>(dd + off) + ip; };
      record_event(c, E[0]);
      CKL(launch_slice_rows(reinterpret_cast<SliceRowsDesc*>(dd + o_sa) + i, pre(o_sap), nw, sapre[ip + nw], c->stream));
      record_event(c, E[1]);
      CKL(launch_gemm_bf16s(reinterpret_cast<OzGemmDesc*>(dd + o_g1) + i, pre(o_g1p), nw, g1pre[ip + nw],
                            c->opt.max_spin, derr, bn1, ns, c->stream));
      record_event(c, E[2]);
      if (spmm_bw)
        CKL(launch_spmm_df_smem(reinterpret_cast<SpmmDfDesc*>(dd + o_sp) + i, pre(o_spp), nw, sppre[ip + nw], spmm_bw,
                                max_ncx, c->stream));
      else
        CKL(launch_spmm_df(reinterpret_cast<SpmmDfDesc*>(dd + o_sp) + i, pre(o_spp), nw, sppre[ip + nw], c->stream));
      record_event(c, E[3]);
      CKL(launch_slice_cols(reinterpret_cast<SliceColsDesc*>(dd + o_sb) + i, pre(o_sbp), nw, sbpre[ip + nw], sbmaxk[t],
                            c->stream));
      record_event(c, E[4]);
      CKL(launch_gemm_bf16s(reinterpret_cast<OzGemmDesc*>(dd + o_g3) + i, pre(o_g3p), nw, g3pre[ip + nw],
                            c->opt.max_spin, derr, bn3, ns, c->stream));
      record_event(c, E[5]);
      c->launches += 5;
    }
    CKL(launch_extract_df(reinterpret_cast<const float2* const*>(dd + o_env), nw, d_H + p0, d_S + p0, c->stream));
    c->launches += 1;
    std::vector<std::array<int, 3>> reads{{2 + 6 * N, 3 + 6 * N, 10}};
    for (int t = 0; t < N; ++t) {
      const int e = 2 + 6 * t;
      reads.push_back({e, e + 1, 10});
      reads.push_back({e + 1, e + 2, 1});
      reads.push_back({e + 2, e + 3, 2});
      reads.push_back({e + 3, e + 4, 10});
      reads.push_back({e + 4, e + 5, 3});
    }
    site_events(c, fi, p1 == (size_t)np, reads);
    p0 = p1;
  }
  fi.check_err = true;
}


// ----------------------------------------------------------------------------- one matrix-element call
// Everything the call puts on the stream, with no host synchronisation when the
// contraction workspace fits one wave: rotations write capacity-padded states,
// so the contraction is planned from the capacities alone.
// The contraction of the pairs (i, i), which need no rotation, on the side
// stream: stream, workspace and descriptor buffers are swapped for the call and
// profiling events are off.
struct SideScope {
  tnqe_ctx* c;
  explicit SideScope(tnqe_ctx* cc) : c(cc) { swap(); }
  ~SideScope() { swap(); }
  void swap() {
    std::swap(c->stream, c->side);
    std::swap(c->oz_ws, c->oz_ws_side);
    std::swap(c->oz_desc, c->oz_desc_side);
    std::swap(c->con_ws, c->con_ws_side);
    std::swap(c->con_desc, c->con_desc_side);
    std::swap(c->bs_flops, c->bs_flops_side);
    c->no_events = !c->no_events;
  }
};

void ensure_mpo(tnqe_ctx* c, DevMps& m, cudaStream_t st);
void start_mpo(tnqe_ctx* c, DevMps& m);

void enqueue_matrix_elements(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pl, double* dH, double* dS,
                             FinishInfo& fi) {
  const int npairs = (int)pl.size();
  c->launches = 0;
  for (double& x : c->prof) x = 0.0;
  struct PresetReset {
    tnqe_ctx* c;
    ~PresetReset() { c->err_preset = false; }
  } preset_reset{c};
  // Pairs (i, i) need no rotation.  With the sliced path their contraction runs
  // on a second stream while the rotation kernel, which leaves SMs free (one
  // CTA per rotated pair), runs on the first; results are scattered to the
  // caller's order at the end.
  std::vector<int> di, ri;
  for (int p = 0; p < npairs; ++p) (pl[p].first == pl[p].second ? di : ri).push_back(p);
  const bool blocks = c->opt.precision == TNQE_PREC_FP64 && c->opt.contraction_form == TNQE_FORM_BLOCKS;
  const bool split = (c->opt.precision >= TNQE_PREC_BF16X3 || blocks) && !di.empty() && !ri.empty();
  std::vector<std::pair<int, int>> pr;
  double *oH = dH, *oS = dS;
  if (split) {
    if (!c->side) {
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CK(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, lo));
      CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
    c->split_out.ensure(sizeof(double) * 2 * npairs);
    c->split_idx.ensure(sizeof(int) * npairs);
    oH = c->split_out.as<double>();
    oS = oH + npairs;
    std::vector<int> order(di);
    order.insert(order.end(), ri.begin(), ri.end());
    upload(c, c->split_idx.p, order.data(), sizeof(int) * npairs);
    c->tc_err.ensure(256);
    CK(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
    c->err_preset = true;
    CK(cudaEventRecord(c->ev_fork, c->stream));
    for (int p : ri) pr.push_back(pl[p]);
  }
  const std::vector<std::pair<int, int>>& pm = split ? pr : pl;
  const int nm = (int)pm.size();
  double* mH = split ? oH + di.size() : dH;
  double* mS = split ? oS + di.size() : dS;
  record_event(c, c->ev[0]);
  RotBatch rb;
  run_rotations(c, pm, rb, 1);
  for (const auto& p : pl) start_mpo(c, *c->mps[p.first]);   // builds not yet started run beside the rotation
  record_event(c, c->ev[1]);
  // The bra states' MPOs: their host builds started just above; the host
  // waits for them here, while the rotation kernel runs, and uploads them (on
  // the side stream when the (i, i) pairs contract there).
  {
    std::vector<int> bras;
    for (const auto& p : pl)
      if (!c->mps[p.first]->mpo_ready) bras.push_back(p.first);
    std::sort(bras.begin(), bras.end());
    bras.erase(std::unique(bras.begin(), bras.end()), bras.end());
    if (!bras.empty()) {
      if (split) {
        if (!c->ev_mpo) CK(cudaEventCreateWithFlags(&c->ev_mpo, cudaEventDisableTiming));
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      }
      for (int i : bras) ensure_mpo(c, *c->mps[i], split ? c->side : c->stream);
      if (split) {
        CK(cudaEventRecord(c->ev_mpo, c->side));
        CK(cudaStreamWaitEvent(c->stream, c->ev_mpo, 0));
      }
    }
  }
  if (split) {
    // submitted after the rotation kernel, so that its CTAs take their SMs first
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    std::vector<std::pair<int, int>> pd;
    std::vector<KetView> kd;
    for (int p : di) {
      pd.push_back(pl[p]);
      const DevMps& mi = *c->mps[pl[p].first];
      kd.push_back(KetView{mi.d_t, mi.off, mi.dims, mi.d_sec});
    }
    {
      FinishInfo fs;
      SideScope scope(c);
      if (blocks) run_contractions_bs(c, pd, kd, oH, oS, fs);
      else run_contractions_oz(c, pd, kd, oH, oS, fs);
      if (!fs.single_wave) fi.single_wave = false;
      fi.bs_flops.insert(fi.bs_flops.end(), fs.bs_flops.begin(), fs.bs_flops.end());
    }
    CK(cudaEventRecord(c->ev_join, c->side));
  }
  std::vector<KetView> kets(nm);
  for (int p = 0; p < nm; ++p) {
    const DevMps& mi = *c->mps[pm[p].first];
    kets[p].base = mi.d_t;
    kets[p].off = mi.off;
    kets[p].dims = mi.dims;
    kets[p].sec = mi.d_sec;
  }
  for (size_t k = 0; k < rb.pair_idx.size(); ++k) {
    KetView& kv = kets[rb.pair_idx[k]];
    kv.base = rb.work[k];
    kv.off = rb.woff[k];
    kv.dims = rb.cap[k];
    kv.sec = rb.sec[k];
  }
  record_event(c, c->ev[2]);
  if (blocks) run_contractions_bs(c, pm, kets, mH, mS, fi);
  else if (c->opt.precision == TNQE_PREC_TF32X3) run_contractions_tc(c, pm, kets, mH, mS, fi);
  else if (c->opt.precision >= TNQE_PREC_BF16X3) run_contractions_oz(c, pm, kets, mH, mS, fi);
  else run_contractions(c, pm, kets, mH, mS, fi);
  record_event(c, c->ev[3]);
  if (split) {
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    CKL(launch_scatter_pairs(oH, oS, c->split_idx.as<int>(), npairs, dH, dS, c->stream));
    c->launches += 1;
  }
  fi.nrot = (int)rb.pair_idx.size();
  if (fi.nrot) {
    fi.rot_small = c->rot_small.as<unsigned char>();
    fi.per_small = rb.per_small;
    fi.o_stat = rb.o_stat;
    fi.o_flops = rb.o_flops;
    fi.ev_reads.push_back({0, 1, 0});
  }
  fi.pstat.assign(c->prof, c->prof + TNQE_PROFILE_LEN);
  fi.launches = c->launches;
}

// After the stream has drained: rotation status and FLOPs, event timings, errors.
void finish_matrix_elements(tnqe_ctx* c, const FinishInfo& fi) {
  for (int k = 0; k < TNQE_PROFILE_LEN; ++k) c->prof[k] = fi.pstat.empty() ? 0.0 : fi.pstat[k];
  c->launches = fi.launches;
  int st = 0;
  if (fi.nrot) {
    std::vector<unsigned char> small(fi.per_small * fi.nrot);
    CK(cudaMemcpy(small.data(), fi.rot_small, small.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < fi.nrot; ++k) {
      int s1 = 0;
      double f1 = 0.0;
      std::memcpy(&s1, small.data() + fi.per_small * k + fi.o_stat, sizeof(int));
      std::memcpy(&f1, small.data() + fi.per_small * k + fi.o_flops, sizeof(double));
      st |= s1;
      c->prof[4] += f1;
    }
  }
  for (const double* f : fi.bs_flops) {
    double h[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(h, f, sizeof(h), cudaMemcpyDeviceToHost));
    c->prof[5] += h[0];
    c->prof[8] += h[1];
    c->prof[7] += h[2];
  }
  for (const auto& r : fi.ev_reads) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->pev[r[0]], c->pev[r[1]]));
    c->prof[r[2]] += ms;
  }
  float t01 = 0, t23 = 0, t03 = 0;
  CK(cudaEventElapsedTime(&t01, c->ev[0], c->ev[1]));
  CK(cudaEventElapsedTime(&t23, c->ev[2], c->ev[3]));
  CK(cudaEventElapsedTime(&t03, c->ev[0], c->ev[3]));
  c->times[0] = t01;
  c->times[1] = t23;
  c->times[2] = t03;
  if (fi.check_err) {
    int herr = 0;
    CK(cudaMemcpy(&herr, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) throw Error(TNQE_ERR_TIMEOUT, "a tensor-core pipeline wait ran out of iterations");
  }
  if (st & STATUS_OVERFLOW) throw Error(TNQE_ERR_STATE, "rotation scratch overflow");
  if (st & STATUS_NOCONV)
    throw Error(TNQE_ERR_NOCONV, "Jacobi SVD hit the sweep limit on a " + std::to_string((st >> 8) & 4095) + " x " +
                                     std::to_string((st >> 20) & 4095) + " block (results written)");
}

std::vector<long long> graph_key(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pl) {
  long long cut = 0;
  static_assert(sizeof(double) == sizeof(long long), "");
  std::memcpy(&cut, &c->opt.cutoff, sizeof(cut));
  std::vector<long long> k{c->generation, c->opt.precision, c->opt.contraction_form, c->opt.chi_rot, cut,
                           c->opt.renormalize_rotated,
                           c->opt.max_jacobi_sweeps, c->opt.max_spin, c->tune.oz_bn1, c->tune.oz_bn3,
                           c->tune.spmm_bw, c->tune.bs_t1, c->tune.bs_t2, c->tune.bs_t3, (long long)pl.size()};
  for (const auto& p : pl) k.push_back((long long)p.first * 65536 + p.second);
  return k;
}

// Record the call into a CUDA graph for later replays.  The eager run that just
// finished sized every workspace, so planning allocates nothing here; if it
// would (or anything else fails), the capture is dropped and calls stay eager.
void capture_matrix_elements(tnqe_ctx* c, const std::vector<std::pair<int, int>>& pl, const std::vector<long long>& key,
                             double* dH, double* dS) {
  double prof_keep[TNQE_PROFILE_LEN];
  std::copy(c->prof, c->prof + TNQE_PROFILE_LEN, prof_keep);
  const int launches_keep = c->launches;
  auto ge = std::make_unique<GraphEntry>();
  const unsigned long long epoch0 = g_alloc_epoch.load();
  bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    c->capturing = true;
    c->cap_uploads = &ge->uploads;
    try {
      enqueue_matrix_elements(c, pl, dH, dS, ge->fin);
    } catch (const Error&) {
      ok = false;
    }
    c->capturing = false;
    c->cap_uploads = nullptr;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    ok = ok && e == cudaSuccess && g != nullptr && g_alloc_epoch.load() == epoch0;
    // per-node priorities: the rotation kernel keeps its launch priority in the replays
    if (ok) ok = cudaGraphInstantiate(&ge->exec, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();   // a failed capture leaves no sticky error behind
  std::copy(prof_keep, prof_keep + TNQE_PROFILE_LEN, c->prof);
  c->launches = launches_keep;
  if (!ok) return;
  ge->epoch = epoch0;
  if (c->graphs.size() >= 16) c->graphs.erase(c->graphs.begin());
  c->graphs[key] = std::move(ge);
}

void check_ctx(tnqe_ctx* c) {
  if (!c) throw Error(TNQE_ERR_ARG, "null context");
  CK(cudaSetDevice(c->opt.device));
}

// ----------------------------------------------------------------------------- add_mps validation
// Host part of adding a state: validate it (orthogonal U, bond dimensions,
// particle-number block structure, (n_alpha, n_beta) sector, left-orthonormal
// sites 0..N-2), sort every bond by charge and lay the tensors out in that
// order (host, back to back; offsets in m.off).  Throws Error(TNQE_ERR_ARG).
// Run f(0..n-1) on up to 8 host threads (static interleaved shares).
template <class F> void parallel_for(int n, F f) {
  const int nt = std::max(1, std::min({n, 8, (int)std::thread::hardware_concurrency()}));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

// A state's site tensors on the host, sorted by charge, one allocation without
// initialisation (every entry is written).
struct HostTensor {
  std::unique_ptr<double[]> p;
  double* ext = nullptr;                 // a caller's buffer of ext_cap doubles, used when it is large enough
  size_t ext_cap = 0;
  size_t n = 0;
  double* data() { return ext && ext_cap >= n ? ext : p.get(); }
};

void order_mps_host(int N, int na, int nb, const double* const* tensors, const int* bond_dims, const double* U,
                    DevMps& m, HostTensor& out) {
  if (!tensors || !bond_dims || !U) throw Error(TNQE_ERR_ARG, "null argument");
  if (bond_dims[0] != 1 || bond_dims[N] != 1) throw Error(TNQE_ERR_ARG, "bond_dims[0] and bond_dims[N] must be 1");
  for (int b = 0; b <= N; ++b)
    if (bond_dims[b] < 1 || bond_dims[b] > 256) throw Error(TNQE_ERR_ARG, "bond dimensions must be in [1, 256]");
  // U orthogonal
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      double acc = 0.0;
      for (int a = 0; a < N; ++a) acc += U[(size_t)a * N + p] * U[(size_t)a * N + q];
      if (std::fabs(acc - (p == q ? 1.0 : 0.0)) > 1e-12) throw Error(TNQE_ERR_ARG, "U is not orthogonal to 1e-12");
    }
  m.U.assign(U, U + (size_t)N * N);
  // charges of every bond index, left to right.  The charge of right index r is
  // that of the first row (l, k) with weight in column r; the scan of a site
  // stops once every column has one, and the parallel pass below checks every
  // weighted entry against the charges.  The tolerance of a site is 1e-12 of
  // its largest entry.
  std::vector<double> amax(N, 0.0);
  for (int s = 0; s < N; ++s)
    if (!tensors[s]) throw Error(TNQE_ERR_ARG, "null site tensor");
  parallel_for(N, [&](int s) {
    const double* A = tensors[s];
    const long long n = (long long)bond_dims[s] * 4 * bond_dims[s + 1];
    double mx = 0.0;
    for (long long x = 0; x < n; ++x) mx = std::max(mx, std::fabs(A[x]));
    amax[s] = mx;
  });
  std::vector<std::vector<int>> q(N + 1);
  q[0] = {0};
  int noweight = -1;
  for (int s = 0; s < N; ++s) {
    const int cl = bond_dims[s], cr = bond_dims[s + 1];
    const double* A = tensors[s];
    const double tol = 1e-12 * amax[s];
    q[s + 1].assign(cr, -1);
    int missing = cr;
    for (int l = 0; l < cl && missing > 0; ++l)
      for (int k = 0; k < 4 && missing > 0; ++k) {
        const int qlk = (q[s][l] / QSTRIDE + (k & 1)) * QSTRIDE + q[s][l] % QSTRIDE + (k >> 1);
        const double* row = A + ((size_t)l * 4 + k) * cr;
        for (int r = 0; r < cr; ++r)
          if (q[s + 1][r] < 0 && std::fabs(row[r]) > tol) {
            q[s + 1][r] = qlk;
            --missing;
          }
      }
    if (missing > 0) {                            // reported below, after the block checks of the sites before
      noweight = s;
      break;
    }
  }
  // the block-structure checks of the sites whose charges are known (all of
  // them unless a bond index has no weight), then the errors in site order
  const int nok = noweight >= 0 ? noweight : N;
  std::vector<int> bad_block(N, 0);
  parallel_for(nok, [&](int s) {
    const int cl = bond_dims[s], cr = bond_dims[s + 1];
    const double* A = tensors[s];
    const double tol = 1e-12 * amax[s];
    const std::vector<int>& qr0 = q[s + 1];
    for (int l = 0; l < cl && !bad_block[s]; ++l)
      for (int k = 0; k < 4; ++k) {
        const int qlk = (q[s][l] / QSTRIDE + (k & 1)) * QSTRIDE + q[s][l] % QSTRIDE + (k >> 1);
        const double* row = A + ((size_t)l * 4 + k) * cr;
        for (int r = 0; r < cr; ++r)
          if (std::fabs(row[r]) > tol && qr0[r] != qlk) bad_block[s] = 1;
      }
  });
  for (int s = 0; s < nok; ++s)
    if (bad_block[s])
      throw Error(TNQE_ERR_ARG, "site " + std::to_string(s) + ": entry breaks the particle-number block structure");
  if (noweight >= 0)
    throw Error(TNQE_ERR_ARG, "site " + std::to_string(noweight) + ": bond index with no weight");
  if (q[N][0] != na * QSTRIDE + nb) throw Error(TNQE_ERR_ARG, "state is not in the (n_alpha, n_beta) sector");
  // sort every bond by charge (a gauge change: the state is unchanged)
  std::vector<std::vector<int>> perm(N + 1);
  m.dims.assign(bond_dims, bond_dims + N + 1);
  m.sec.assign(N + 1, SectorTable{});
  m.chi = *std::max_element(bond_dims, bond_dims + N + 1);
  for (int b = 0; b <= N; ++b) {
    perm[b].resize(bond_dims[b]);
    for (int x = 0; x < bond_dims[b]; ++x) perm[b][x] = x;
    std::stable_sort(perm[b].begin(), perm[b].end(), [&](int x, int y) { return q[b][x] < q[b][y]; });
    SectorTable& T = m.sec[b];
    T.nsec = 0;
    for (int x = 0; x < bond_dims[b]; ++x) {
      const int qq = q[b][perm[b][x]];
      if (T.nsec == 0 || T.q[T.nsec - 1] != qq) {
        if (T.nsec >= MAXSEC) throw Error(TNQE_ERR_ARG, "too many charge sectors on one bond");
        T.q[T.nsec] = qq;
        T.off[T.nsec] = x;
        T.dim[T.nsec] = 0;
        ++T.nsec;
      }
      ++T.dim[T.nsec - 1];
    }
  }
  m.off.assign(N, 0);
  size_t total = 0;
  for (int s = 0; s < N; ++s) {
    m.off[s] = (long long)total;
    total += (size_t)bond_dims[s] * 4 * bond_dims[s + 1];
  }
  out.n = total;
  if (!(out.ext && out.ext_cap >= total)) out.p.reset(new double[total]);   // every entry is written below
  // one pass per site, sites on host threads: sites 0..N-2 left-orthonormal (the Gram matrix of the
  // columns, block by block: columns of different charge have disjoint support);
  // the site written in the sorted order, zero outside the blocks
  std::vector<int> bad_orth(N, 0);
  parallel_for(N, [&](int s) {
    const int cl = bond_dims[s], cr = bond_dims[s + 1];
    const double* A = tensors[s];
    const std::vector<int>& qr0 = q[s + 1];
    if (s + 1 < N) {
      std::vector<double> gram((size_t)cr * cr, 0.0);
      std::vector<std::vector<int>> same(cr);      // columns of r's charge at or after r
      for (int r1 = 0; r1 < cr; ++r1)
        for (int r2 = r1; r2 < cr; ++r2)
          if (qr0[r1] == qr0[r2]) same[r1].push_back(r2);
      for (int lk = 0; lk < cl * 4; ++lk) {
        const double* row = A + (size_t)lk * cr;
        for (int r1 = 0; r1 < cr; ++r1) {
          const double a1 = row[r1];
          if (a1 == 0.0) continue;
          double* g = gram.data() + (size_t)r1 * cr;
          for (int r2 : same[r1]) g[r2] += a1 * row[r2];
        }
      }
      for (int r1 = 0; r1 < cr && !bad_orth[s]; ++r1)
        for (int r2 : same[r1])
          if (std::fabs(gram[(size_t)r1 * cr + r2] - (r1 == r2 ? 1.0 : 0.0)) > 1e-10) bad_orth[s] = 1;
    }
    std::vector<int> qr(cr);
    for (int r = 0; r < cr; ++r) qr[r] = qr0[perm[s + 1][r]];
    const int* pr = perm[s + 1].data();
    double* dst0 = out.data() + m.off[s];
    for (int l = 0; l < cl; ++l) {
      const int ql = q[s][perm[s][l]];
      for (int k = 0; k < 4; ++k) {
        const int qlk = (ql / QSTRIDE + (k & 1)) * QSTRIDE + ql % QSTRIDE + (k >> 1);
        const double* src = A + ((size_t)perm[s][l] * 4 + k) * cr;
        double* dst = dst0 + ((size_t)l * 4 + k) * cr;
        for (int r = 0; r < cr; ++r) dst[r] = (qlk == qr[r]) ? src[pr[r]] : 0.0;   // below-tolerance noise outside the blocks
      }
    }
  });
  for (int s = 0; s + 1 < N; ++s)
    if (bad_orth[s]) throw Error(TNQE_ERR_ARG, "site " + std::to_string(s) + " is not left-orthonormal");
}

// The Hamiltonian MPO of one state's basis, built on a host thread and packed
// for one upload: the CSR of every site in FP64, FP32 and double-float, the row
// order by nonzero count, and the charge classes of channels and rows.
struct MpoPack {
  Mpo mpo;
  BlockTables bt;
  HostPack pk;
  std::vector<size_t> o_choff, o_chd, o_chw, o_rcoff, o_rcd, o_rcrows, o_rcnnz;
  std::vector<size_t> o_rowptr, o_col, o_val, o_perm, o_v32, o_vdf, o_ent;
};

std::shared_ptr<MpoPack> build_mpo_pack(const double* h1, const double* eri, const std::vector<double>& U, int N) {
  auto P = std::make_shared<MpoPack>();
  std::vector<double> hU, gU;
  rotate_integrals(h1, eri, U.data(), N, hU, gU);
  P->mpo = build_mpo(hU.data(), gU.data(), N);
  if (P->mpo.dims[N] != 2) throw Error(TNQE_ERR_STATE, "MPO construction failed");
  P->bt = block_tables(P->mpo, N);
  const BlockTables& bt = P->bt;
  HostPack& pk = P->pk;
  P->o_choff.resize(N + 1);
  P->o_chd.resize(N + 1);
  P->o_chw.resize(N + 1);
  for (int b = 0; b <= N; ++b) {
    P->o_choff[b] = pk.add(bt.ch_off[b]);
    P->o_chd[b] = pk.add(bt.ch_d[b]);
    P->o_chw[b] = pk.add(bt.ch_w[b]);
  }
  for (auto* v : {&P->o_rcoff, &P->o_rcd, &P->o_rcrows, &P->o_rcnnz, &P->o_rowptr, &P->o_col, &P->o_val, &P->o_perm,
                  &P->o_v32, &P->o_vdf, &P->o_ent})
    v->resize(N);
  for (int t = 0; t < N; ++t) {
    P->o_rcoff[t] = pk.add(bt.rc_off[t]);
    P->o_rcd[t] = pk.add(bt.rc_d[t]);
    P->o_rcrows[t] = pk.add(bt.rc_rows[t]);
    P->o_rcnnz[t] = pk.add(bt.rc_nnz[t]);
  }
  for (int t = 0; t < N; ++t) {
    const MpoSite& S = P->mpo.sites[t];
    P->o_rowptr[t] = pk.add(S.rowptr);
    P->o_col[t] = pk.add(S.col);
    P->o_val[t] = pk.add(S.val);
    {
      const std::vector<int>& rp = S.rowptr;
      std::vector<int> perm(rp.size() - 1);
      for (size_t r = 0; r < perm.size(); ++r) perm[r] = (int)r;
      std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
      P->o_perm[t] = pk.add(perm);
    }
    std::vector<float> v32(S.val.begin(), S.val.end());
    P->o_v32[t] = pk.add(v32);
    std::vector<float2> vdf(v32.size());
    for (size_t e = 0; e < v32.size(); ++e) {
      const double v = S.val[e];
      vdf[e].x = (float)v;
      vdf[e].y = (float)(v - (double)vdf[e].x);
    }
    P->o_vdf[t] = pk.add(vdf);
    std::vector<float4> ent(vdf.size());
    for (size_t e = 0; e < vdf.size(); ++e) {
      int col = S.col[e];
      float cf;
      std::memcpy(&cf, &col, sizeof(cf));
      ent[e] = make_float4(vdf[e].x, vdf[e].y, cf, 0.f);
    }
    P->o_ent[t] = pk.add(ent);
  }
  return P;
}

// Host part of tnqe_add_mps: validate and order the state, upload its tensors
// (one allocation, one copy) and start the build of its MPO on a host thread.
// Start the host build of state m's MPO (once).  The first call that needs it
// starts it, after its rotation kernel is enqueued, so that the builds run
// beside the rotation and not beside the host work of the following
// tnqe_add_mps calls (N = 14, chi = 128, 16 states: 55 -> 34 ms of adds).
void start_mpo(tnqe_ctx* c, DevMps& m) {
  if (m.mpo_ready || m.mpo_future.valid()) return;
  m.mpo_future = std::async(std::launch::async, build_mpo_pack, c->h1.data(), c->eri.data(), std::cref(m.U), c->N);
}

void prepare_mps(tnqe_ctx* c, const double* const* tensors, const int* bond_dims, const double* U, DevMps& m) {
  const int N = c->N;
  // the sorted tensors go to a pinned staging buffer of the context (grown when
  // too small), so that the upload is one direct copy
  size_t need = 0;
  for (int s = 0; bond_dims && s < N; ++s)      // (order_mps_host reports bad arguments)
    need += (size_t)std::min(std::max(bond_dims[s], 0), 256) * 4 * std::min(std::max(bond_dims[s + 1], 0), 256);
  if (need > c->stage_cap) {
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (cudaHostAlloc(&c->stage, need * sizeof(double), cudaHostAllocDefault) == cudaSuccess) c->stage_cap = need;
    else c->stage = nullptr;                    // pageable memory then
  }
  HostTensor host;
  host.ext = static_cast<double*>(c->stage);
  host.ext_cap = c->stage_cap;
  order_mps_host(N, c->na, c->nb, tensors, bond_dims, U, m, host);
  HostPack pk;                                   // the small arrays, behind the tensors
  const size_t o_off = pk.add(m.off), o_dims = pk.add(m.dims), o_sec = pk.add(m.sec);
  const size_t tbytes = (host.n * sizeof(double) + 255) & ~(size_t)255;
  void* dev = nullptr;
  CK(cudaMalloc(&dev, tbytes + pk.h.size()));
  m.owned.push_back(dev);
  unsigned char* base = static_cast<unsigned char*>(dev);
  CK(cudaMemcpy(base, host.data(), host.n * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(base + tbytes, pk.h.data(), pk.h.size(), cudaMemcpyHostToDevice));
  base += tbytes;
  m.d_t = reinterpret_cast<double*>(static_cast<unsigned char*>(dev));
  m.d_off = reinterpret_cast<long long*>(base + o_off);
  m.d_dims = reinterpret_cast<int*>(base + o_dims);
  m.d_sec = reinterpret_cast<SectorTable*>(base + o_sec);
}

// The MPO of state m on the device: wait for its host build (if still running)
// and upload it with one asynchronous copy on `st`.
void ensure_mpo(tnqe_ctx* c, DevMps& m, cudaStream_t st) {
  if (m.mpo_ready) return;
  start_mpo(c, m);
  if (c->capturing) throw Error(TNQE_ERR_STATE, "MPO upload inside a graph capture");
  std::shared_ptr<MpoPack> P;
  try {
    P = m.mpo_future.get();
  } catch (const Error&) {
    throw;
  } catch (const std::exception& e) {
    throw Error(TNQE_ERR_NOMEM, std::string("MPO build failed: ") + e.what());
  }
  const int N = c->N;
  void* dev = nullptr;
  CK(cudaMalloc(&dev, P->pk.h.size()));
  m.owned.push_back(dev);
  CK(cudaMemcpyAsync(dev, P->pk.h.data(), P->pk.h.size(), cudaMemcpyHostToDevice, st));
  unsigned char* base = static_cast<unsigned char*>(dev);
  const BlockTables& bt = P->bt;
  for (int b = 0; b <= N; ++b) {
    BsChannels ch{};
    ch.ncls = (int)bt.ch_off[b].size() - 1;
    ch.off = reinterpret_cast<const int*>(base + P->o_choff[b]);
    ch.d = reinterpret_cast<const int*>(base + P->o_chd[b]);
    ch.w = reinterpret_cast<const int*>(base + P->o_chw[b]);
    m.bs_ch.push_back(ch);
  }
  for (int t = 0; t < N; ++t) {
    BsRows r{};
    r.ncls = (int)bt.rc_off[t].size() - 1;
    r.off = reinterpret_cast<const int*>(base + P->o_rcoff[t]);
    r.d = reinterpret_cast<const int*>(base + P->o_rcd[t]);
    r.rows = reinterpret_cast<const int*>(base + P->o_rcrows[t]);
    r.nnz = reinterpret_cast<const int*>(base + P->o_rcnnz[t]);
    m.bs_rows.push_back(r);
  }
  for (int t = 0; t < N; ++t) {
    m.d_rowptr.push_back(reinterpret_cast<int*>(base + P->o_rowptr[t]));
    m.d_col.push_back(reinterpret_cast<int*>(base + P->o_col[t]));
    m.d_val.push_back(reinterpret_cast<double*>(base + P->o_val[t]));
    m.d_rowperm.push_back(reinterpret_cast<int*>(base + P->o_perm[t]));
    m.d_val32.push_back(reinterpret_cast<float*>(base + P->o_v32[t]));
    m.d_valdf.push_back(reinterpret_cast<float2*>(base + P->o_vdf[t]));
    m.d_ent.push_back(reinterpret_cast<float4*>(base + P->o_ent[t]));
  }
  m.mpo = std::move(P->mpo);
  m.mpo_ready = true;
}

// The class of a pair list for the tuning cache: N (which fixes the MPO bond
// dimensions), precision and form, and the multiset of (bra bond dimension,
// ket bond dimension) over the pairs (the largest over the bonds of each state).
std::string tune_key(tnqe_ctx* c, const int* pairs, int npairs) {
  std::map<std::array<int, 2>, int> cls;
  const int M = (int)c->mps.size();
  for (int p = 0; p < npairs; ++p) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    if (i < 0 || j < 0 || i >= M || j >= M) throw Error(TNQE_ERR_STATE, "unknown MPS id");
    const DevMps& a = *c->mps[i];
    const DevMps& b = *c->mps[j];
    const int da = *std::max_element(a.dims.begin(), a.dims.end());
    const int db = *std::max_element(b.dims.begin(), b.dims.end());
    ++cls[{da, db}];
  }
  std::string k = "N=" + std::to_string(c->N) + " prec=" + std::to_string(c->opt.precision) +
                  " form=" + std::to_string(c->opt.contraction_form);
  for (const auto& kv : cls)
    k += " " + std::to_string(kv.first[0]) + "x" + std::to_string(kv.first[1]) + "*" + std::to_string(kv.second);
  return k;
}

// One line per tuned class: "tnqe-tune <key> | bs_t1 bs_t2 bs_t3 oz_bn1 oz_bn3 spmm_bw".
bool tune_cache_lookup(tnqe_ctx* c, const std::string& key) {
  FILE* f = std::fopen(c->tune_cache.c_str(), "r");
  if (!f) return false;
  const std::string head = "tnqe-tune " + key + " |";
  char buf[8192];
  bool found = false;
  while (std::fgets(buf, sizeof(buf), f)) {
    std::string line(buf);
    if (line.compare(0, head.size(), head) != 0) continue;
    int v[6];
    if (std::sscanf(line.c_str() + head.size(), "%d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) != 6)
      continue;
    const bool ok = (v[0] == 64 || v[0] == 128 || v[0] == 256) && (v[1] == 64 || v[1] == 128 || v[1] == 256) &&
                    (v[2] == 64 || v[2] == 128 || v[2] == 256) && (v[3] == 64 || v[3] == 128) &&
                    (v[4] == 64 || v[4] == 128) && v[5] >= 0 && v[5] <= 8 && !(v[5] & (v[5] - 1));
    if (!ok) continue;
    c->tune.bs_t1 = v[0];
    c->tune.bs_t2 = v[1];
    c->tune.bs_t3 = v[2];
    c->tune.oz_bn1 = v[3];
    c->tune.oz_bn3 = v[4];
    c->tune.spmm_bw = v[5];
    found = true;                                  // the last matching line wins
  }
  std::fclose(f);
  return found;
}

void tune_cache_store(tnqe_ctx* c, const std::string& key) {
  FILE* f = std::fopen(c->tune_cache.c_str(), "a");
  if (!f) throw Error(TNQE_ERR_ARG, "cannot append to the autotune cache " + c->tune_cache);
  std::fprintf(f, "tnqe-tune %s | %d %d %d %d %d %d\n", key.c_str(), c->tune.bs_t1, c->tune.bs_t2, c->tune.bs_t3,
               c->tune.oz_bn1, c->tune.oz_bn3, c->tune.spmm_bw);
  std::fclose(f);
}

}  // namespace

// ============================================================================= ABI
extern "C" {

void tnqe_default_options(tnqe_options* o) {
  if (!o) return;
  o->precision = TNQE_PREC_FP64;
  o->chi_rot = 0;
  o->cutoff = 1e-14;
  o->solve_eps = 1e-10;
  o->renormalize_rotated = 0;
  o->max_jacobi_sweeps = 60;
  o->max_spin = 1LL << 26;
  o->cuda_stream = nullptr;
  o->device = 0;
  o->use_graphs = 1;
  o->contraction_form = TNQE_FORM_BLOCKS;
  o->autotune_cache = nullptr;
  o->workspace_limit = 0;
}

tnqe_status tnqe_givens_host(const double* V, int N, int* site, int* side, double* c, double* s, int cap,
                             int* ngates, int* neg_site) {
  try {
    if (!V || !ngates || !neg_site || N < 1 || N > 64) return TNQE_ERR_ARG;
    const tnqe::GivensPlan P = tnqe::givens_plan(V, N);
    *ngates = (int)P.gates.size();
    *neg_site = P.neg_site;
    if (!site || !side || !c || !s) return TNQE_OK;
    if (cap < (int)P.gates.size()) return TNQE_ERR_ARG;
    for (size_t g = 0; g < P.gates.size(); ++g) {
      site[g] = P.gates[g].site;
      side[g] = P.gates[g].side;
      c[g] = P.gates[g].c;
      s[g] = P.gates[g].s;
    }
    return TNQE_OK;
  } catch (...) {
    return TNQE_ERR_NOMEM;
  }
}

tnqe_status tnqe_gate_host(double c, double s, double* G) {
  if (!G || !(std::fabs(c * c + s * s - 1.0) < 1e-12)) return TNQE_ERR_ARG;
  tnqe::gate_matrix(c, s, G);
  return TNQE_OK;
}

tnqe_status tnqe_rotate_integrals_host(const double* h1, const double* eri, const double* U, int N, double* h_out,
                                       double* eri_out) {
  try {
    if (!h1 || !eri || !U || !h_out || !eri_out || N < 1 || N > 64) return TNQE_ERR_ARG;
    std::vector<double> h, g;
    tnqe::rotate_integrals(h1, eri, U, N, h, g);
    std::copy(h.begin(), h.end(), h_out);
    std::copy(g.begin(), g.end(), eri_out);
    return TNQE_OK;
  } catch (...) {
    return TNQE_ERR_NOMEM;
  }
}

tnqe_status tnqe_check_mps(int N, int n_alpha, int n_beta, const double* const* tensors, const int* bond_dims,
                           const double* U, char* msg, int msg_len) {
  auto put = [&](const std::string& t) {
    if (msg && msg_len > 0) {
      const size_t n = std::min(t.size(), (size_t)msg_len - 1);
      std::memcpy(msg, t.data(), n);
      msg[n] = 0;
    }
  };
  try {
    if (N < 1 || N > 32 || n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N) {
      put("bad N or electron numbers");
      return TNQE_ERR_ARG;
    }
    DevMps m;
    HostTensor host;
    order_mps_host(N, n_alpha, n_beta, tensors, bond_dims, U, m, host);
    put("");
    return TNQE_OK;
  } catch (const Error& e) {
    put(e.what());
    return e.st;
  } catch (const std::bad_alloc&) {
    put("out of host memory");
    return TNQE_ERR_NOMEM;
  }
}

tnqe_status tnqe_mpo_host(const double* h1, const double* eri, int N, int* dims, long long* nnz, int* rowptr,
                          int* col, double* val, long long cap) {
  try {
    if (!h1 || !eri || !dims || !nnz || N < 1 || N > 32) return TNQE_ERR_ARG;
    const tnqe::Mpo m = tnqe::build_mpo(h1, eri, N);
    long long total = 0;
    for (int b = 0; b <= N; ++b) dims[b] = m.dims[b];
    for (int t = 0; t < N; ++t) {
      nnz[t] = (long long)m.sites[t].val.size();
      total += nnz[t];
    }
    if (!rowptr || !col || !val) return TNQE_OK;
    if (cap < total) return TNQE_ERR_ARG;
    long long ro = 0, eo = 0;
    for (int t = 0; t < N; ++t) {
      const tnqe::MpoSite& S = m.sites[t];
      std::copy(S.rowptr.begin(), S.rowptr.end(), rowptr + ro);
      std::copy(S.col.begin(), S.col.end(), col + eo);
      std::copy(S.val.begin(), S.val.end(), val + eo);
      ro += (long long)S.rowptr.size();
      eo += (long long)S.val.size();
    }
    return TNQE_OK;
  } catch (const std::bad_alloc&) {
    return TNQE_ERR_NOMEM;
  } catch (...) {
    return TNQE_ERR_STATE;
  }
}

tnqe_status tnqe_create(const double* h1, const double* eri, int N, int n_alpha, int n_beta,
                        const tnqe_options* opt, tnqe_ctx** out) {
  if (!out) return TNQE_ERR_ARG;
  *out = nullptr;
  tnqe_ctx* c = nullptr;
  try {
    if (!h1 || !eri) throw Error(TNQE_ERR_ARG, "null integrals");
    if (N < 1 || N > 32) throw Error(TNQE_ERR_ARG, "N must be in [1, 32]");
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N || n_alpha > 14 || n_beta > 14)
      throw Error(TNQE_ERR_ARG, "electron counts must be in [0, min(N, 14)]");
    c = new tnqe_ctx();
    if (opt) c->opt = *opt; else tnqe_default_options(&c->opt);
    if (c->opt.autotune_cache) c->tune_cache = c->opt.autotune_cache;
    c->opt.autotune_cache = nullptr;                 // the context keeps its own copy
    if (c->opt.precision < 0 || c->opt.precision > TNQE_PREC_BF16X15) throw Error(TNQE_ERR_ARG, "unknown precision");
    if (c->opt.contraction_form != TNQE_FORM_BLOCKS && c->opt.contraction_form != TNQE_FORM_DENSE)
      throw Error(TNQE_ERR_ARG, "unknown contraction form");
    c->N = N;
    c->na = n_alpha;
    c->nb = n_beta;
    c->h1.assign(h1, h1 + (size_t)N * N);
    c->eri.assign(eri, eri + (size_t)N * N * N * N);
    c->exact_dim.assign(N + 1, 0);
    for (int b = 0; b <= N; ++b) {
      double tot = 0.0;
      for (int a = 0; a <= std::min(b, n_alpha); ++a)
        for (int bb = 0; bb <= std::min(b, n_beta); ++bb) {
          if (n_alpha - a > N - b || n_beta - bb > N - b) continue;
          tot += std::min(binom(b, a) * binom(b, bb), binom(N - b, n_alpha - a) * binom(N - b, n_beta - bb));
        }
      c->exact_dim[b] = (int)std::min(tot, 1e9);
    }
    CK(cudaSetDevice(c->opt.device));
    if (c->opt.cuda_stream) {
      c->stream = (cudaStream_t)c->opt.cuda_stream;
    } else {
      CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    for (auto& e : c->ev) CK(cudaEventCreate(&e));
    c->pev.assign(4 + 6 * N, nullptr);
    for (auto& e : c->pev) CK(cudaEventCreate(&e));
    *out = c;
    return TNQE_OK;
  } catch (const Error& e) {
    if (c) tnqe_destroy(c);
    return e.st;
  } catch (...) {
    if (c) tnqe_destroy(c);
    return TNQE_ERR_NOMEM;
  }
}

tnqe_status tnqe_add_mps(tnqe_ctx* c, const double* const* tensors, const int* bond_dims, const double* U,
                         int* mps_id) {
  try {
    check_ctx(c);
    auto m = std::make_unique<DevMps>();
    try {
      prepare_mps(c, tensors, bond_dims, U, *m);
    } catch (...) {
      m->free_all();
      throw;
    }
    c->mps.push_back(std::move(m));
    ++c->generation;
    clear_graphs(c);
    if (mps_id) *mps_id = (int)c->mps.size() - 1;
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::exception& e) {
    return fail(c, Error(TNQE_ERR_NOMEM, e.what()));
  }
}

tnqe_status tnqe_reset_mps(tnqe_ctx* c) {
  try {
    check_ctx(c);
    CK(cudaStreamSynchronize(c->stream));
    clear_graphs(c);
    ++c->generation;
    for (auto& m : c->mps) m->free_all();
    c->mps.clear();
    c->plans.clear();
    for (void* p : c->plan_arenas) cudaFree(p);
    c->plan_arenas.clear();
    c->kept_pair_valid = 0;
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_rotate(tnqe_ctx* c, int i, int j, double* discarded_weight) {
  try {
    check_ctx(c);
    const int M = (int)c->mps.size();
    if (i < 0 || j < 0 || i >= M || j >= M) throw Error(TNQE_ERR_STATE, "unknown MPS id");
    c->launches = 0;
    const int N = c->N;
    if (i == j) {
      c->kept_dims = c->mps[j]->dims;
      c->kept_off = c->mps[j]->off;
      c->kept_pair_valid = 2 + j;          // the unrotated state j
      if (discarded_weight) *discarded_weight = 0.0;
      return TNQE_OK;
    }
    RotBatch rb;
    run_rotations(c, {{i, j}}, rb, 0);
    std::vector<std::vector<int>> dims;
    std::vector<double> disc;
    int st = 0;
    fetch_rotation_results(c, rb, dims, disc, st);
    c->kept_dims = dims[0];
    c->kept_off = rb.woff[0];
    c->kept_pair_valid = 1;
    if (discarded_weight) *discarded_weight = disc[0];
    (void)N;
    if (st & STATUS_OVERFLOW) throw Error(TNQE_ERR_STATE, "rotation scratch overflow");
    if (st & STATUS_NOCONV) throw Error(TNQE_ERR_NOCONV, "Jacobi SVD hit the sweep limit");
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_get_rotated(tnqe_ctx* c, int* bond_dims, double* tensors, long long max_doubles) {
  try {
    check_ctx(c);
    if (!c->kept_pair_valid) throw Error(TNQE_ERR_STATE, "no rotated state kept");
    const int N = c->N;
    long long need = 0;
    for (int s = 0; s < N; ++s) need += (long long)c->kept_dims[s] * 4 * c->kept_dims[s + 1];
    if (bond_dims) std::memcpy(bond_dims, c->kept_dims.data(), sizeof(int) * (N + 1));
    if (!tensors) return TNQE_OK;
    if (max_doubles < need) throw Error(TNQE_ERR_ARG, "output buffer too small");
    const double* base = c->kept_pair_valid == 1 ? c->rot_work.as<double>() : c->mps[c->kept_pair_valid - 2]->d_t;
    long long o = 0;
    for (int s = 0; s < N; ++s) {
      const long long n = (long long)c->kept_dims[s] * 4 * c->kept_dims[s + 1];
      CK(cudaMemcpyAsync(tensors + o, base + c->kept_off[s], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
      o += n;
    }
    CK(cudaStreamSynchronize(c->stream));
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_matrix_elements(tnqe_ctx* c, const int* pairs, int npairs, double* H_out, double* S_out) {
  try {
    check_ctx(c);
    if (npairs < 0 || (npairs > 0 && (!pairs || !H_out || !S_out))) throw Error(TNQE_ERR_ARG, "bad pair list");
    if (npairs == 0) return TNQE_OK;
    const int M = (int)c->mps.size();
    std::vector<std::pair<int, int>> pl(npairs);
    for (int p = 0; p < npairs; ++p) {
      const int i = pairs[2 * p], j = pairs[2 * p + 1];
      if (i < 0 || j < 0 || i >= M || j >= M) throw Error(TNQE_ERR_STATE, "unknown MPS id in pair list");
      pl[p] = {i, j};
    }
    c->kept_pair_valid = 0;
    c->con_out.ensure(sizeof(double) * 2 * npairs);
    double* dH = c->con_out.as<double>();
    double* dS = dH + npairs;
    GraphEntry* ge = nullptr;
    std::vector<long long> key;
    if (c->opt.use_graphs) {
      key = graph_key(c, pl);
      auto it = c->graphs.find(key);
      if (it != c->graphs.end() && it->second->epoch == g_alloc_epoch.load()) ge = it->second.get();
    }
    FinishInfo fi;
    if (ge) {
      for (const Upload& u : ge->uploads)
        CK(cudaMemcpyAsync(u.dst, u.data.data(), u.data.size(), cudaMemcpyHostToDevice, c->stream));
      CK(cudaGraphLaunch(ge->exec, c->stream));
      fi = ge->fin;
    } else {
      enqueue_matrix_elements(c, pl, dH, dS, fi);
    }
    const bool hdev = is_device_ptr(H_out), sdev = is_device_ptr(S_out);
    CK(cudaMemcpyAsync(H_out, dH, sizeof(double) * npairs, hdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(S_out, dS, sizeof(double) * npairs, sdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    finish_matrix_elements(c, fi);
    if (c->opt.use_graphs && !ge && fi.single_wave) {
      if (c->seen.size() > 64) c->seen.clear();
      if (c->seen[key]++ >= 1) capture_matrix_elements(c, pl, key, dH, dS);
    }
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::exception& e) {
    return fail(c, Error(TNQE_ERR_NOMEM, e.what()));
  }
}

tnqe_status tnqe_autotune(tnqe_ctx* c, const int* pairs, int npairs, int* config, double* times) {
  try {
    check_ctx(c);
    if (npairs <= 0 || !pairs) throw Error(TNQE_ERR_ARG, "bad pair list");
    const bool blocks = c->opt.precision == TNQE_PREC_FP64 && c->opt.contraction_form == TNQE_FORM_BLOCKS;
    const bool sliced = c->opt.precision >= TNQE_PREC_BF16X3;
    auto fill_config = [&]() {
      if (!config) return;
      if (blocks) {
        config[0] = c->tune.bs_t1;
        config[1] = c->tune.bs_t2;
        config[2] = c->tune.bs_t3;
      } else {
        config[0] = c->tune.oz_bn1;
        config[1] = c->tune.oz_bn3;
        config[2] = c->tune.spmm_bw;
      }
    };
    if (!blocks && !sliced) {
      fill_config();
      return TNQE_OK;
    }
    const std::string key = tune_key(c, pairs, npairs);
    if (!c->tune_cache.empty() && tune_cache_lookup(c, key)) {   // this class was tuned before
      clear_graphs(c);
      fill_config();
      if (times)
        for (int q = 0; q < 9; ++q) times[q] = 0.0;
      return TNQE_OK;
    }
    struct Cand {
      int a, b, w;
    };
    // charge-block stages: CTA sizes; sliced GEMMs: N tiles of stages 1 and 3 and MPO kernel width
    const Cand bcands[3] = {{64, 64, 64}, {128, 128, 128}, {256, 256, 256}};
    const Cand ocands[3] = {{128, 128, 8}, {64, 64, 4}, {128, 128, 2}};
    const Cand* cands = blocks ? bcands : ocands;
    const int keep_graphs = c->opt.use_graphs;
    c->opt.use_graphs = 0;
    std::vector<double> Hh(npairs), Sh(npairs);
    double t[3][3];
    tnqe_status st = TNQE_OK;
    auto apply = [&](const Cand& x) {
      if (blocks) {
        c->tune.bs_t1 = x.a;
        c->tune.bs_t3 = x.b;
        c->tune.bs_t2 = x.w;
      } else {
        c->tune.oz_bn1 = x.a;
        c->tune.oz_bn3 = x.b;
        c->tune.spmm_bw = x.w;
      }
    };
    for (int k = 0; k < 3 && st == TNQE_OK; ++k) {
      apply(cands[k]);
      for (int rep = 0; rep < 2 && st == TNQE_OK; ++rep)   // the first run warms allocations and caches
        st = tnqe_matrix_elements(c, pairs, npairs, Hh.data(), Sh.data());
      t[k][0] = c->prof[1];
      t[k][1] = c->prof[3];
      t[k][2] = c->prof[2];
      if (times)
        for (int q = 0; q < 3; ++q) times[3 * k + q] = t[k][q];
    }
    c->opt.use_graphs = keep_graphs;
    if (st != TNQE_OK) return st;
    int b1 = 0, b3 = 0, bw = 0;
    for (int k = 1; k < 3; ++k) {
      if (t[k][0] < t[b1][0]) b1 = k;
      if (t[k][1] < t[b3][1]) b3 = k;
      if (t[k][2] < t[bw][2]) bw = k;
    }
    apply(Cand{cands[b1].a, cands[b3].b, cands[bw].w});
    CK(cudaStreamSynchronize(c->stream));
    clear_graphs(c);
    if (!c->tune_cache.empty()) tune_cache_store(c, key);
    fill_config();
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_set_block_tuning(tnqe_ctx* c, int t1, int t2, int t3) {
  if (!c) return TNQE_ERR_ARG;
  for (int t : {t1, t2, t3})
    if (t != 64 && t != 128 && t != 256) {
      c->err = "charge-block stage CTA sizes must be 64, 128 or 256";
      return TNQE_ERR_ARG;
    }
  c->tune.bs_t1 = t1;
  c->tune.bs_t2 = t2;
  c->tune.bs_t3 = t3;
  clear_graphs(c);
  return TNQE_OK;
}

tnqe_status tnqe_set_tuning(tnqe_ctx* c, int bn1, int bn3, int spmm_bw) {
  if (!c) return TNQE_ERR_ARG;
  if ((bn1 != 64 && bn1 != 128) || (bn3 != 64 && bn3 != 128) || spmm_bw < 0 || spmm_bw > 8 ||
      (spmm_bw & (spmm_bw - 1))) {
    c->err = "tile choices: bn1, bn3 in {64, 128}; spmm_bw in {0, 1, 2, 4, 8}";
    return TNQE_ERR_ARG;
  }
  c->tune.oz_bn1 = bn1;
  c->tune.oz_bn3 = bn3;
  c->tune.spmm_bw = spmm_bw;
  return TNQE_OK;
}

tnqe_status tnqe_clear_graphs(tnqe_ctx* c) {
  try {
    check_ctx(c);
    CK(cudaStreamSynchronize(c->stream));
    clear_graphs(c);
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

int tnqe_graph_count(const tnqe_ctx* c) { return c ? (int)c->graphs.size() : 0; }

tnqe_status tnqe_solve_ex(tnqe_ctx* c, const double* H, const double* S, int M, double eps, double* E, double* C,
                          int* rank_kept, double* kappa1) {
  try {
    check_ctx(c);
    if (M < 1 || M > 32 || !H || !S || !E || !C || !rank_kept || !kappa1) throw Error(TNQE_ERR_ARG, "bad solve arguments");
    if (!(eps >= 0.0) || eps >= 1.0) throw Error(TNQE_ERR_ARG, "eps must be in [0, 1)");
    const size_t mm = (size_t)M * M;
    c->solve_buf.ensure(sizeof(double) * (3 * 32 * 32 + 32 + 2) + 16);   // sized for M = 32 once
    double* dH = c->solve_buf.as<double>();
    double* dS = dH + mm;
    double* dC = dS + mm;
    double* dE = dC + mm;
    double* dK = dE + M;
    int* dR = reinterpret_cast<int*>(dK + 1);
    int* dSt = dR + 1;
    CK(cudaMemcpyAsync(dH, H, sizeof(double) * mm, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dS, S, sizeof(double) * mm, cudaMemcpyHostToDevice, c->stream));
    CKL(launch_solve(dH, dS, M, eps, c->opt.max_jacobi_sweeps, dE, dC, dR, dK, dSt, c->stream));
    int st = 0;
    CK(cudaMemcpyAsync(E, dE, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(C, dC, sizeof(double) * mm, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(rank_kept, dR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(kappa1, dK, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&st, dSt, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st) throw Error(TNQE_ERR_NOCONV, "eigensolver hit the sweep limit");
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_solve(tnqe_ctx* c, const double* H, const double* S, int M, double* E, double* C, int* rank_kept,
                       double* kappa1) {
  if (!c) return TNQE_ERR_ARG;
  return tnqe_solve_ex(c, H, S, M, c->opt.solve_eps, E, C, rank_kept, kappa1);
}

tnqe_status tnqe_dependence(tnqe_ctx* c, const double* S, int M, double eps, double* residuals) {
  try {
    check_ctx(c);
    if (M < 1 || M > 32 || !S || !residuals) throw Error(TNQE_ERR_ARG, "bad dependence arguments");
    if (!(eps >= 0.0) || eps >= 1.0) throw Error(TNQE_ERR_ARG, "eps must be in [0, 1)");
    const size_t mm = (size_t)M * M;
    c->solve_buf.ensure(sizeof(double) * (3 * 32 * 32 + 32 + 2) + 16);
    double* dS = c->solve_buf.as<double>();
    double* dR = dS + mm;
    int* dSt = reinterpret_cast<int*>(dR + M);
    CK(cudaMemcpyAsync(dS, S, sizeof(double) * mm, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(dSt, 0, sizeof(int), c->stream));
    CKL(launch_dependence(dS, M, eps, c->opt.max_jacobi_sweeps, dR, dSt, c->stream));
    int st = 0;
    CK(cudaMemcpyAsync(residuals, dR, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&st, dSt, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st) throw Error(TNQE_ERR_NOCONV, "eigensolver hit the sweep limit");
    return TNQE_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

tnqe_status tnqe_set_precision(tnqe_ctx* c, int precision) {
  if (!c) return TNQE_ERR_ARG;
  if (precision < 0 || precision > TNQE_PREC_BF16X15) {
    c->err = "unknown precision";
    return TNQE_ERR_ARG;
  }
  c->opt.precision = precision;
  return TNQE_OK;
}

tnqe_status tnqe_set_form(tnqe_ctx* c, int form) {
  if (!c) return TNQE_ERR_ARG;
  if (form != TNQE_FORM_BLOCKS && form != TNQE_FORM_DENSE) {
    c->err = "unknown contraction form";
    return TNQE_ERR_ARG;
  }
  c->opt.contraction_form = form;
  return TNQE_OK;
}

tnqe_status tnqe_last_timing(const tnqe_ctx* c, double* times, int* launches) {
  if (!c) return TNQE_ERR_ARG;
  if (times)
    for (int k = 0; k < 3; ++k) times[k] = c->times[k];
  if (launches) *launches = c->launches;
  return TNQE_OK;
}

tnqe_status tnqe_last_profile(const tnqe_ctx* c, double* prof, int n) {
  if (!c || !prof || n < 0) return TNQE_ERR_ARG;
  for (int k = 0; k < n && k < TNQE_PROFILE_LEN; ++k) prof[k] = c->prof[k];
  if (n > 9) prof[9] = c->launches;
  return TNQE_OK;
}

const char* tnqe_last_error(const tnqe_ctx* c) { return c ? c->err.c_str() : "null context"; }

void tnqe_destroy(tnqe_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->opt.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& m : c->mps) m->free_all();
  for (void* p : c->plan_arenas) cudaFree(p);
  c->rot_work.release();
  c->rot_scratch.release();
  c->rot_meta.release();
  c->rot_small.release();
  c->rot_desc.release();
  if (c->stage) cudaFreeHost(c->stage);
  c->stage = nullptr;
  c->con_ws.release();
  c->con_desc.release();
  c->con_out.release();
  c->tc_ws.release();
  c->tc_desc.release();
  c->tc_err.release();
  c->oz_ws.release();
  c->oz_desc.release();
  c->oz_ws_side.release();
  c->oz_desc_side.release();
  c->split_out.release();
  c->split_idx.release();
  c->con_ws_side.release();
  c->con_desc_side.release();
  c->bs_flops.release();
  c->bs_flops_side.release();
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_mpo) cudaEventDestroy(c->ev_mpo);
  if (c->side) cudaStreamDestroy(c->side);
  c->solve_buf.release();
  c->graphs.clear();
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->pev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
