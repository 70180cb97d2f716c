// C ABI of the batched R-MATEX library: setup (ordering, factorisation,
// schedules, upload) and the run loop that drives the CUDA kernels.
//
// Run structure (Alg. 2 for every group at once, one group per column):
//   round r = segment r of every group that has one.  Per round:
//     inputs   z = G^{-1} B u(l), z' = G^{-1} B s, w = G^{-1} C z'   (Eq. 5/6)
//     start    v = x + F = x - z + w, beta = ||v||                   (Alg. 1)
//     Arnoldi  w = (C + gamma G)^{-1} C v_j, two Gram-Schmidt passes, residual
//              test of Sec. 3.3.3 per column; converged columns retire
//     outputs  y(t_o) = beta e^{(t_o - l) H_m} e_1,  X[o] += V y + z + h z' - w
//     hand-off x(l_{j+1}) for the next round.
// After the first (plain) run the same pass is recorded as a CUDA graph and
// replayed while the device's active-column counts match the recording.
// Also here: batches of contexts as one graph, the trapezoidal baseline, the
// other Krylov spaces' operators, and the allocation-free solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <new>
#include <string>
#include <vector>

#include "../../include/matex.h"
#include "internal.h"
#include "kernels.h"

using namespace matex;

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Round {
  int32_t begin;  // first column record
  int32_t K;      // columns
  int32_t obeg_min, oend_max;
  double cover = 0.0;          // share of (column, output) pairs of the range the columns hold
  int32_t ev_begin = 0, nev = 0;  // -P events of the round (recombine_p)
};

// Device address of the allocation-free solve's static scratch array on
// device `dev` (defined with matex_solve_noalloc below).
matex_status noalloc_scratch(int dev, void** out, std::string& err);

// Launch and sweep counts of one pass of the run.
struct PassCounts {
  int launches = 0, sweepsM = 0, sweepsG = 0, tc_rounds = 0;
  int64_t solve_cols = 0;
};

}  // namespace

struct matex_ctx {
  std::string err;
  cudaStream_t st = nullptr;
  int device = 0;
  // problem
  int64_t n = 0;
  int32_t n_src = 0, n_groups = 0, m_max = 0, n_times = 0;
  double gamma = 0, tol = 0, dt_out = 0, T = 0;
  matex_opts opts{};
  std::vector<int32_t> rows;      // output rows (original numbering); empty = all
  std::vector<int32_t> replay;    // per segment, empty = adaptive
  std::vector<int32_t> sel_groups;
  int64_t n_segments = 0;
  int32_t nrows_out = 0;
  std::vector<double> pwl_v_host_shape;  // length of pwl_v
  // structure
  Symbolic S;
  std::vector<LevelPlan> levels;
  SplitScratch split;              // chunked reductions of the level launches
  // resident rounds (opts.resident): per-level work lists, the choice, and
  // the setup's timings of one solve pair both ways (ms, -1 if not taken)
  // wide supernodes on the tensor cores (opts.tc_solve): the level plans
  // without their split tasks, per level their (supernode, row tile) lists,
  // the panel slices and row scales of both factors and directions, the
  // and per column count whether a call uses them
  int ts_minw = 0;
  std::vector<LevelPlan> levels_n;
  std::vector<TsLevel> ts_levels;
  TsSup* ts_sups = nullptr;
  int ts_n = 0;
  __nv_bfloat16* tsA[2][2] = {};   // [factor M, G][forward, backward]
  double* tsR[2][2] = {};
  int ts_mtf = 0, ts_mtb = 0;      // most row tiles of a wide supernode, per direction
  std::vector<int8_t> ts_by_ncols;
  int ts_min_cols = 0;
  ResidentPlan rplan;
  ResFactor rM, rG;          // the factors' resident copies
  ResStoreSup* rsup = nullptr;
  bool resident_ok = false;  // plan built and shared-memory limits set
  bool resident = false;
  float res_pair_ms = -1.f, lvl_pair_ms = -1.f;
  // resident rounds: every column record's z' and w, solved ahead of the
  // rounds in one launch per run (null: each round kernel solves its own)
  double *pre_zp = nullptr, *pre_w = nullptr;
  // single-column level kernels (opts.single_column): their plan and whether
  // solves of one column take them
  K1Plan k1;
  std::vector<int32_t> k1_fw_off, k1_bw_off;
  bool k1_use = false;
  TcScratch tc;                    // tensor-core recombination (kdim_cap 0: not used)
  int32_t *ev_o_d = nullptr, *ev_q_d = nullptr;  // -P events of all rounds
  // persistent solve: per column count (1..ldy) one PersistLevel row per level
  PersistLevel* plev_d = nullptr;
  std::vector<long long> pf_total, pb_total;   // per column count
  unsigned long long* pcounters = nullptr;     // ticket, then fdone[nsup], bdone[nsup]
  int* fpend = nullptr;
  int* fpend_init = nullptr;
  int32_t *sup_level_d = nullptr, *nft_d = nullptr, *nbt_d = nullptr;
  size_t psmem = 0;
  int pgrid = 0;
  bool inject_wait = false;  // test hook: a dependency that never completes
  // autotuned solve launch mode per column count (0 persistent, 1 per level)
  std::vector<int8_t> mode_by_ncols;
  std::vector<int32_t> tune_reps, tune_modes;
  std::vector<float> level_tune_ms;  // per level and direction: best time of the chosen block
  std::vector<float> tune_ms;
  // adjoint tape (opts.tape): per record (non-zero segment) basis slot = record
  int64_t n_records = 0;
  bool taped = false;        // a run with the tape has completed
  double *TA = nullptr, *TZp = nullptr, *THt = nullptr, *Tbeta = nullptr;
  // adjoint work
  double *AW = nullptr, *XBg = nullptr, *CARRYg = nullptr, *CBg = nullptr;
  double *YBO = nullptr, *YOUT = nullptr, *YBL = nullptr, *YL = nullptr, *HTB = nullptr;
  double *BETAB = nullptr, *D1 = nullptr, *HD = nullptr, *D0 = nullptr, *S1 = nullptr, *S2 = nullptr;
  int32_t *iota_d = nullptr, *mrec_d = nullptr, *act_d = nullptr;
  // checkpointed adjoint (opts.tape = 2): windows of tape_W rounds, recompute
  // blocks of tape_Kb groups; CK holds {x, z} of every column of each
  // window's first round, window w's from slot ck_base[w]
  int tape_W = 0, tape_Kb = 0;
  int64_t tape_bytes = 0;
  std::vector<int64_t> ck_base;
  double* CK = nullptr;
  std::vector<int32_t> h_group_all;
  std::vector<Round> rounds;          // batched: segment r of every group per round
  // Batches of groups run one after another, each with its own rounds and
  // initial states; per-group state and basis slots are reused from batch to
  // batch (state slot = rc_group, source group = rc_sgroup).  One batch with
  // slot = group except for ramp columns beyond kRampBatch, which hand no
  // state to later segments.
  struct Batch { int32_t r0, r1, i0, ni; };  // rounds [r0, r1), initial states [i0, i0 + ni)
  std::vector<Batch> batches;
  int32_t g_slots = 1;                // per-group state and basis slots
  int32_t* rc_sgroup = nullptr;
  int32_t* init_slots_d = nullptr;    // state slot of each entry of init_groups
  std::vector<Round> serial_rounds;   // one group at a time: one column per round
  bool serial = false;
  std::vector<int32_t> serial_cover;
  matex_stats setup_stats{};
  matex_stats last{};
  // device memory
  std::vector<void*> allocs;
  DevFactor fM{}, fG{};
  SourceTable src{};
  double* c_perm = nullptr;
  double* dc_perm = nullptr;
  int32_t* perm = nullptr;      // new -> old
  int32_t* out_map = nullptr;   // output row r -> new index
  int32_t* sel_groups_d = nullptr;
  double* pwl_v_d = nullptr;
  double* pwl_base_d = nullptr;  // the currents given at setup (amplitude scale 1)
  std::vector<double> c_host;    // capacitances, original order (refactorisation)
  std::vector<int64_t> g_rowptr_h;
  std::vector<int32_t> g_col_h;
  std::vector<double> g_val_h;
  // round tables
  int32_t *rc_group = nullptr, *rc_seg = nullptr, *rc_obeg = nullptr, *rc_nout = nullptr;
  int32_t* rc_vslot = nullptr;
  double *rc_l0 = nullptr, *rc_len = nullptr, *rc_hfirst = nullptr, *rc_lprev = nullptr;
  std::vector<int32_t> init_groups;   // groups whose input is non-zero at t = 0
  int32_t* init_groups_d = nullptr;
  // zero pattern of the setup currents, per selected group: the local
  // transition spots, which segments were skipped as identically zero, and
  // whether the current at t = 0 is non-zero (checked by set_sources)
  std::vector<int32_t> pwl_off_h;
  std::vector<double> pwl_t_h;
  std::vector<std::vector<int32_t>> gsrc_h;
  std::vector<std::vector<double>> glts_h;
  std::vector<std::vector<char>> gzero_h;
  std::vector<char> ginit_h;
  int64_t* rc_segid = nullptr;
  int32_t* replay_d = nullptr;
  // work buffers
  int ldy = 8;
  int Kmax = 1;
  int nchunks = 1;
  double* Y = nullptr;
  double* Y2 = nullptr;     // forward-solve intermediate, same shape as Y
  double* Vb = nullptr;     // [n_groups][kMaxB][n]
  double *Zb = nullptr, *Zpb = nullptr, *Wb = nullptr, *Xb = nullptr;  // [n_groups][n]
  double* Xp = nullptr;     // [n_times][n]
  double* xdc = nullptr;    // [n]
  double* partials = nullptr;
  SmallState ss{};
  int32_t *iterA = nullptr, *iterB = nullptr, *iter_grp = nullptr, *d_count = nullptr;
  int32_t* h_count = nullptr;  // pinned
  double* coef = nullptr;
  double* yend = nullptr;
  int32_t* tcut = nullptr;   // [Kmax][2] tail cut of each column (tail_eps > 0)
  double* pbound = nullptr;  // [Kmax][2] bounds on the column's -P term (tail_eps > 0)
  int32_t *m_rec = nullptr, *st_rec = nullptr;
  double* out_buf = nullptr;   // device output for matex_run_host
  // host copies of the round tables (profiling arithmetic)
  std::vector<int32_t> h_nout_all;
  std::vector<int64_t> h_segid_all;
  std::vector<int32_t> round_cover;  // outputs covered per round
  int64_t offd_rows = 0;              // sum over supernodes of off-diagonal rows
  // CUDA graph of one run: recorded after a plain run, replayed while the
  // device's active-column counts equal the recorded ones
  std::vector<int32_t> kit_trace;  // counts read by the host in the plain run, in order
  cudaStream_t gst = nullptr;      // private capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  PassCounts graph_counts;
  double graph_ms = 0.0;
  int64_t graph_gen = 0;           // bumped at every new recording
  // trapezoidal baseline (matex_tr_run): factor of C + h/2 G for the last h
  // (structure shared with the C + gamma G factor), G in CSR in the permuted
  // order, state and input vectors, and the recorded loop
  double tr_h = 0.0;
  DevFactor fT{};
  int64_t* trG_rowptr = nullptr;
  int32_t* trG_col = nullptr;
  double* trG_val = nullptr;
  double *trX = nullptr, *trB0 = nullptr, *trB1 = nullptr;
  cudaGraphExec_t tr_exec = nullptr;
  int tr_substeps = 0;            // substeps the recorded loop was built for
  double tr_factor_ms = 0.0;
  // profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Pending { int cls, e0; int64_t launches; double flops, bytes; int round; };
  std::vector<Pending> pend;
  matex_profile prof{};

  ~matex_ctx() {
    for (void* p : allocs) cudaFree(p);
    if (h_count) cudaFreeHost(h_count);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (tr_exec) cudaGraphExecDestroy(tr_exec);
    if (graph) cudaGraphDestroy(graph);
    if (gst) cudaStreamDestroy(gst);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }

  template <typename T>
  bool alloc(T*& p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(q);
    p = static_cast<T*>(q);
    return true;
  }
  template <typename T>
  bool upload(T*& p, const T* h, size_t count) {
    if (!alloc(p, count)) return false;
    if (count && cudaMemcpy(p, h, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
    return true;
  }
};

namespace {

matex_status fail(matex_ctx* c, matex_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

matex_status cuda_check(matex_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, MATEX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return MATEX_OK;
}

thread_local std::string g_setup_err;

int roundup8(int x) { return (x + 7) & ~7; }

// Value of one PWL source at time x: held before the first and after the last
// breakpoint, linear in between (the same rule as the device evaluation).
double pwl_value(const double* t, const double* v, int np, double x) {
  if (x <= t[0]) return v[0];
  if (x >= t[np - 1]) return v[np - 1];
  int j = 0;
  while (j + 1 < np && t[j + 1] <= x) ++j;
  return (v[j + 1] - v[j]) / (t[j + 1] - t[j]) * (x - t[j]) + v[j];
}

// True when every source of the group injects exactly zero at time x.
bool group_input_zero(const std::vector<int32_t>& srcs, const int32_t* pwl_off, const double* pwl_t,
                      const double* pwl_v, double x) {
  for (int32_t s : srcs) {
    const int o = pwl_off[s], np = pwl_off[s + 1] - o;
    if (pwl_value(pwl_t + o, pwl_v + o, np, x) != 0.0) return false;
  }
  return true;
}

// Local transition spots of one group: its sources' breakpoints inside (0, T)
// plus 0 and T, sorted and unique (Sec. 3.1).
std::vector<double> group_lts(const std::vector<int32_t>& srcs, const int32_t* pwl_off,
                              const double* pwl_t, double T) {
  std::vector<double> pts = {0.0, T};
  for (int32_t s : srcs)
    for (int32_t p = pwl_off[s]; p < pwl_off[s + 1]; ++p)
      if (pwl_t[p] > 0.0 && pwl_t[p] < T) pts.push_back(pwl_t[p]);
  std::sort(pts.begin(), pts.end());
  pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
  return pts;
}

// Ramp decomposition (Sec. 3.1's source decomposition carried to single
// ramps).  On [0, T] a PWL source equals its value at 0 plus, at each of its
// breakpoints tau in (0, T), ds max(0, t - tau) with ds the change of slope
// at tau, plus a ramp at tau = 0 with the slope right of 0.  Each (group,
// kind, tau) with kind 0 = starting values, 1 = ramp becomes a group; groups
// are ordered by (group, kind, tau), their sources by original index.  A
// ramp source's PWL is (tau, 0), (T, ds (T - tau)); a starting value's is
// (0, u(0)).
struct RampProblem {
  std::vector<int32_t> node, off, grp;
  std::vector<double> t, v;
  int32_t ngroups = 0;
};

double slope_right(const double* t, const double* v, int np, double x) {
  if (x < t[0] || x >= t[np - 1]) return 0.0;
  const int j = (int)(std::upper_bound(t, t + np, x) - t) - 1;
  return (v[j + 1] - v[j]) / (t[j + 1] - t[j]);
}

double slope_left(const double* t, const double* v, int np, double x) {
  if (x <= t[0] || x > t[np - 1]) return 0.0;
  const int j = (int)(std::lower_bound(t, t + np, x) - t) - 1;
  return (v[j + 1] - v[j]) / (t[j + 1] - t[j]);
}

void ramp_transform(int32_t n_src, const int32_t* src_node, const int32_t* pwl_off,
                    const double* pwl_t, const double* pwl_v, const int32_t* src_group, double T,
                    RampProblem& out) {
  struct E {
    int32_t k, kind;
    double tau;
    int32_t s;
    int npts;
    double t0, v0, t1, v1;
  };
  std::vector<E> es;
  for (int32_t s = 0; s < n_src; ++s) {
    const int o = pwl_off[s], np = pwl_off[s + 1] - o;
    const double* t = pwl_t + o;
    const double* v = pwl_v + o;
    const int32_t k = src_group[s];
    const double u0 = pwl_value(t, v, np, 0.0);
    if (u0 != 0.0) es.push_back(E{k, 0, 0.0, s, 1, 0.0, u0, 0.0, 0.0});
    const double s0 = slope_right(t, v, np, 0.0);
    if (s0 != 0.0) es.push_back(E{k, 1, 0.0, s, 2, 0.0, 0.0, T, s0 * T});
    for (int j = 0; j < np; ++j) {
      const double tau = t[j];
      if (!(tau > 0.0 && tau < T)) continue;
      const double ds = slope_right(t, v, np, tau) - slope_left(t, v, np, tau);
      if (ds != 0.0) es.push_back(E{k, 1, tau, s, 2, tau, 0.0, T, ds * (T - tau)});
    }
  }
  std::stable_sort(es.begin(), es.end(), [](const E& a, const E& b) {
    if (a.k != b.k) return a.k < b.k;
    if (a.kind != b.kind) return a.kind < b.kind;
    return a.tau < b.tau;
  });
  out = RampProblem();
  out.off.push_back(0);
  for (size_t i = 0; i < es.size(); ++i) {
    const E& e = es[i];
    if (i == 0 || e.k != es[i - 1].k || e.kind != es[i - 1].kind || e.tau != es[i - 1].tau)
      out.ngroups++;
    out.node.push_back(src_node[e.s]);
    out.grp.push_back(out.ngroups - 1);
    out.t.push_back(e.t0);
    out.v.push_back(e.v0);
    if (e.npts == 2) {
      out.t.push_back(e.t1);
      out.v.push_back(e.v1);
    }
    out.off.push_back((int32_t)out.t.size());
  }
}

// Per tree level: forward tasks (supernode, 32 panel rows), backward tasks
// (supernode, 32 panel columns) and the column block.  Returns false on an
// allocation failure.
constexpr int kSolveSmemCap = 24 * 1024 + 512;  // keeps ~8 solve CTAs resident per SM
constexpr int kSplitFor = 4;                    // threads sharing one panel row / column
constexpr int kSolveThreadsFor = 128;           // threads of a solve CTA (partial sums per thread)

bool plan_levels(matex_ctx* c) {
  const Symbolic& S = c->S;
  const int nlev = (int)S.level_ptr.size() - 1;
  c->levels.resize(nlev);
  std::vector<int2> ft, bt;
  std::vector<int32_t> pack;
  std::vector<char> fpacked(S.nsup, 0), bpacked(S.nsup, 0);
  std::vector<size_t> fofs(nlev + 1), bofs(nlev + 1);
  int smem_need = 0;
  // small supernodes of a level share one task: forward packs rows of panels
  // at most 16 wide, backward packs columns of panels at most 16 wide and 64
  // rows long (a longer panel keeps the 4-thread split dot of its own task)
  constexpr int kPackLd = 384;
  int dev_sms = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int kPackTarget = 8 * std::max(dev_sms, 1);  // CTAs that keep every SM busy
  std::vector<int32_t> pack_a, pack_b;  // per entry: rows / columns of the earlier entries
  auto flush = [&](std::vector<int32_t>& cur, std::vector<int2>& out, int mode) {
    if (cur.empty()) return;
    out.push_back(make_int2(-1 - (int)pack.size(), (int)cur.size() | mode));
    int a = 0, b = 0;
    for (int32_t s : cur) {
      pack.push_back(s);
      pack_a.push_back(a);
      pack_b.push_back(b);
      a += (int)(S.sup_rowptr[s + 1] - S.sup_rowptr[s]);
      b += S.sup_first[s + 1] - S.sup_first[s];
    }
    cur.clear();
  };
  auto sup_w = [&](int s) { return S.sup_first[s + 1] - S.sup_first[s]; };
  auto sup_ld = [&](int s) { return (int)(S.sup_rowptr[s + 1] - S.sup_rowptr[s]); };
  for (int l = 0; l < nlev; ++l) {
    LevelPlan& L = c->levels[l];
    fofs[l] = ft.size();
    bofs[l] = bt.size();
    int mw = 1, mwr = 1;
    bool any_bpack = false;
    std::vector<int32_t> cur;
    int rows = 0;
    // packed tasks run one thread per row (forward) or column (backward), and a
    // warp takes as long as its longest thread: packing the level's supernodes
    // in order of width (forward) or panel length (backward) keeps the threads
    // of a warp alike
    std::vector<int32_t> by_w(S.level_sups.begin() + S.level_ptr[l],
                              S.level_sups.begin() + S.level_ptr[l + 1]);
    std::vector<int32_t> by_ld = by_w;
    std::stable_sort(by_w.begin(), by_w.end(), [&](int a, int b) { return sup_w(a) > sup_w(b); });
    std::stable_sort(by_ld.begin(), by_ld.end(), [&](int a, int b) { return sup_ld(a) > sup_ld(b); });
    // Packed tasks run their rows (columns) as warp-wide (row, right-hand
    // side) chunks, every lane busy but each warp working through several
    // chunks in turn; or one thread per row, lanes idle where rows of unequal
    // width share a warp but every row at once.  The first wins when the
    // level has enough packed work to fill the GPU, the second when it does
    // not (small grids, upper levels: the solve is then latency-bound).
    int prow = 0, pcol = 0;
    for (const int s : by_w) {
      if (sup_ld(s) <= kPackRows && sup_w(s) <= 16) prow += sup_ld(s);
      if (sup_w(s) <= 16 && sup_ld(s) <= 64) pcol += sup_w(s);
    }
    const int cblocks = std::max(1, c->ldy / 8);
    const int fmode = (prow / kPackRows) * cblocks >= kPackTarget ? 0 : kPackRowwise;
    const int bmode = (pcol / kPackRows) * cblocks >= kPackTarget ? 0 : kPackRowwise;
    L.split_w = L.split_ld = 0;
    for (const int s : by_w) {
      const int w = sup_w(s);
      const int wr = sup_ld(s);
      mw = std::max(mw, w);
      if (!(w <= 16 && wr <= 64)) L.split_ld = std::max(L.split_ld, wr);
      if (wr <= kPackRows && w <= 16) {
        if (rows + wr > kPackRows || (int)cur.size() == kPackMax) { flush(cur, ft, fmode); rows = 0; }
        cur.push_back(s);
        rows += wr;
        fpacked[s] = 1;
      } else {
        mwr = std::max(mwr, wr);
        L.split_w = std::max(L.split_w, w);
        for (int i0 = 0; i0 < wr; i0 += kRowBlock) ft.push_back(make_int2(s, i0));
      }
    }
    flush(cur, ft, fmode);
    int cols = 0, ldsum = 0;
    for (const int s : by_ld) {
      const int w = sup_w(s);
      const int wr = sup_ld(s);
      if (w <= 16 && wr <= 64) {
        if (cols + w > kPackRows || ldsum + wr > kPackLd || (int)cur.size() == kPackMax) {
          flush(cur, bt, bmode);
          cols = ldsum = 0;
        }
        cur.push_back(s);
        cols += w;
        ldsum += wr;
        bpacked[s] = 1;
        any_bpack = true;
      } else {
        mwr = std::max(mwr, wr);
        for (int j0 = 0; j0 < w; j0 += kRowBlock) bt.push_back(make_int2(s, j0));
      }
    }
    flush(cur, bt, bmode);
    // longest tasks first (the block scheduler hands out CTAs in index order,
    // so the level's tail is made of short tasks); duration ~ the length of one
    // thread's dot product: a quarter of the panel extent for split tasks, the
    // whole extent for packed ones (one thread per row or column)
    auto fdur = [&](const int2& t) {
      if (t.x >= 0) return std::min(sup_w(t.x), t.y + kRowBlock) / kSplitFor;
      int d = 0;
      for (int k = 0; k < (t.y & (kPackRowwise - 1)); ++k) d = std::max(d, sup_w(pack[-1 - t.x + k]));
      return d;
    };
    auto bdur = [&](const int2& t) {
      if (t.x >= 0) return (sup_ld(t.x) - t.y) / kSplitFor;
      int d = 0;
      for (int k = 0; k < (t.y & (kPackRowwise - 1)); ++k) d = std::max(d, sup_ld(pack[-1 - t.x + k]));
      return d;
    };
    std::stable_sort(ft.begin() + fofs[l], ft.end(),
                     [&](const int2& a, const int2& b) { return fdur(a) > fdur(b); });
    std::stable_sort(bt.begin() + bofs[l], bt.end(),
                     [&](const int2& a, const int2& b) { return bdur(a) > bdur(b); });
    L.nf = (int32_t)(ft.size() - fofs[l]);
    L.nb = (int32_t)(bt.size() - bofs[l]);
    L.max_w = std::max(mw, kPackRows);
    const int ld_need = std::max(mwr, any_bpack ? kPackLd : 1);
    L.max_wr = ld_need;
    int kb = c->opts.col_block;
    if (kb <= 0) {
      // enough (task, column block) pairs to fill 152 SMs, else narrower blocks
      const int tasks = std::min(L.nf, L.nb * 4);
      kb = tasks >= 512 ? 8 : tasks >= 128 ? 4 : tasks >= 32 ? 2 : 1;
    }
    while (kb > 1 && (size_t)ld_need * kb * sizeof(double) > (size_t)kSolveSmemCap) kb /= 2;
    L.kb = kb;
    L.kbf = L.kbb = kb;
    smem_need = std::max(smem_need, (int)(std::max(std::max(ld_need, L.max_w) * kb,
                                                   kSolveThreadsFor * (kb + 1)) * sizeof(double)));
  }
  fofs[nlev] = ft.size();
  bofs[nlev] = bt.size();
  int2 *fd, *bd;
  int32_t *pk, *pa, *pb;
  if (pack.empty()) {
    pack.push_back(0);
    pack_a.push_back(0);
    pack_b.push_back(0);
  }
  if (!c->upload(fd, ft.data(), ft.size()) || !c->upload(bd, bt.data(), bt.size()) ||
      !c->upload(pk, pack.data(), pack.size()) || !c->upload(pa, pack_a.data(), pack_a.size()) ||
      !c->upload(pb, pack_b.data(), pack_b.size()))
    return false;
  c->fM.pack = c->fG.pack = pk;
  c->fM.pack_a = c->fG.pack_a = pa;
  c->fM.pack_b = c->fG.pack_b = pb;
  for (int l = 0; l < nlev; ++l) {
    c->levels[l].ftasks = fd + fofs[l];
    c->levels[l].btasks = bd + bofs[l];
  }
  if (c->ts_minw > 0) {
    // the same task lists without the split tasks of supernodes at least
    // ts_minw wide (packed tasks hold supernodes at most 16 wide)
    std::vector<int2> ftn, btn;
    std::vector<size_t> fon(nlev + 1), bon(nlev + 1);
    auto narrow = [&](const int2& t) { return t.x < 0 || sup_w(t.x) < c->ts_minw; };
    for (int l = 0; l < nlev; ++l) {
      fon[l] = ftn.size();
      bon[l] = btn.size();
      for (size_t e = fofs[l]; e < fofs[l + 1]; ++e)
        if (narrow(ft[e])) ftn.push_back(ft[e]);
      for (size_t e = bofs[l]; e < bofs[l + 1]; ++e)
        if (narrow(bt[e])) btn.push_back(bt[e]);
    }
    fon[nlev] = ftn.size();
    bon[nlev] = btn.size();
    int2 *fdn = nullptr, *bdn = nullptr;
    if (!c->upload(fdn, ftn.data(), ftn.size()) || !c->upload(bdn, btn.data(), btn.size()))
      return false;
    c->levels_n = c->levels;
    for (int l = 0; l < nlev; ++l) {
      LevelPlan& L = c->levels_n[l];
      L.ftasks = fdn + fon[l];
      L.btasks = bdn + bon[l];
      L.nf = (int32_t)(fon[l + 1] - fon[l]);
      L.nb = (int32_t)(bon[l + 1] - bon[l]);
    }
  }
  set_solve_smem_limit(std::max(smem_need, kSolveSmemTune));
  // persistent schedules for every column count 1..ldy
  std::vector<PersistLevel> pl((size_t)c->ldy * nlev);
  c->pf_total.assign(c->ldy + 1, 0);
  c->pb_total.assign(c->ldy + 1, 0);
  for (int nc = 1; nc <= c->ldy; ++nc) {
    long long fb = 0;
    for (int l = 0; l < nlev; ++l) {
      PersistLevel& P = pl[(size_t)(nc - 1) * nlev + l];
      int kb = c->levels[l].kb;
      while (kb > 1 && kb / 2 >= nc) kb /= 2;
      P.ftasks = fd + fofs[l];
      P.btasks = bd + bofs[l];
      P.nf = c->levels[l].nf;
      P.nb = c->levels[l].nb;
      P.kb = kb;
      P.ncb = (nc + kb - 1) / kb;
      auto batch_for = [](long long tasks) {
        return tasks >= 8192 ? 8 : tasks >= 2048 ? 4 : tasks >= 512 ? 2 : 1;
      };
      P.fbatch = batch_for((long long)P.nf * P.ncb);
      P.bbatch = batch_for((long long)P.nb * P.ncb);
      P.fbase = fb;
      fb += ((long long)P.nf * P.ncb + P.fbatch - 1) / P.fbatch;
    }
    long long bb = 0;
    for (int l = nlev - 1; l >= 0; --l) {
      PersistLevel& P = pl[(size_t)(nc - 1) * nlev + l];
      P.bbase = bb;
      bb += ((long long)P.nb * P.ncb + P.bbatch - 1) / P.bbatch;
    }
    c->pf_total[nc] = fb;
    c->pb_total[nc] = bb;
  }
  if (!c->upload(c->plev_d, pl.data(), pl.size())) return false;
  if (!c->alloc(c->split.part, (size_t)2 * kSplitSlots * kRowBlock * kMaxColBlock) ||
      !c->alloc(c->split.cnt, (size_t)kSplitSlots) ||
      cudaMemset(c->split.cnt, 0, sizeof(int) * kSplitSlots) != cudaSuccess)
    return false;
  std::vector<int32_t> lev(S.nsup), nft(S.nsup), nbt(S.nsup), kids(S.nsup, 0);
  for (int l = 0; l < nlev; ++l)
    for (int k = S.level_ptr[l]; k < S.level_ptr[l + 1]; ++k) lev[S.level_sups[k]] = l;
  for (int32_t s = 0; s < S.nsup; ++s) {
    const int w = S.sup_first[s + 1] - S.sup_first[s];
    const int wr = (int)(S.sup_rowptr[s + 1] - S.sup_rowptr[s]);
    nft[s] = fpacked[s] ? 1 : (wr + kRowBlock - 1) / kRowBlock;
    nbt[s] = bpacked[s] ? 1 : (w + kRowBlock - 1) / kRowBlock;
    if (S.sup_parent[s] >= 0) kids[S.sup_parent[s]]++;
  }
  if (!c->upload(c->sup_level_d, lev.data(), lev.size()) || !c->upload(c->nft_d, nft.data(), nft.size()) ||
      !c->upload(c->nbt_d, nbt.data(), nbt.size()) ||
      !c->upload(c->fpend_init, kids.data(), kids.size()) || !c->alloc(c->fpend, S.nsup) ||
      !c->alloc(c->pcounters, 1 + (size_t)S.nsup))
    return false;
  c->psmem = std::max<size_t>(smem_need, sizeof(double) * 8);
  int bps = persistent_blocks_per_sm(c->psmem);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->pgrid = std::max(1, bps) * std::max(1, sms);
  return true;
}

// The resident rounds' plan blob (see ResidentPlan) and the resident copies
// of both factors: per tree level, leaves first, the panels of its
// supernodes one after another, their forward rows and backward columns in
// supernode order (consecutive threads read consecutive panel entries), the
// level's below-diagonal rows grouped by target row with contributions in
// supernode order, and per level and direction the lanes per dot product.
bool plan_resident(matex_ctx* c, int threads) {
  const Symbolic& S = c->S;
  const int nlev = (int)S.level_ptr.size() - 1;
  if (nlev > kResidentMaxLevels || S.nsup > 65535) return false;
  std::vector<ResSup> sups(S.nsup);
  std::vector<ResStoreSup> store;
  std::vector<int32_t> offs(kResOffN * (nlev + 1), 0), tgt, tpp, tslot, brows;
  std::vector<uint16_t> fsup, bsup;
  struct Upd { int32_t t, ord, slot; };
  std::vector<Upd> up;
  int uslots = 0;
  int64_t dst = 0;
  auto lanes = [&](int items, int longest) {
    // lanes per dot product: the fewest L2 round trips, passes over the
    // level's items times batches of 8 loads per lane (ties: fewer lanes)
    int best = 1;
    long long cost = -1;
    for (int l = 1; l <= 8; l *= 2) {
      const long long passes = ((long long)items * l + threads - 1) / threads;
      const long long batches = (longest + 8LL * l - 1) / (8LL * l);
      if (cost < 0 || passes * batches < cost) {
        cost = passes * batches;
        best = l;
      }
    }
    return best;
  };
  auto at = [&](int seg, int l) -> int32_t& { return offs[seg * (nlev + 1) + l]; };
  for (int l = 0; l <= nlev; ++l) {
    at(kResOffR, l) = (int32_t)fsup.size();
    at(kResOffT, l) = (int32_t)tgt.size();
    at(kResOffC, l) = (int32_t)bsup.size();
    at(kResOffLB, l) = (int32_t)brows.size();
    if (l == nlev) break;
    up.clear();
    int fmax = 1, bmax = 1, rb = 0, cb = 0;
    const int lb = (int)brows.size();
    for (int k = S.level_ptr[l]; k < S.level_ptr[l + 1]; ++k) {
      const int s = S.level_sups[k];
      const int f = S.sup_first[s];
      const int w = S.sup_first[s + 1] - f;
      const int64_t rp = S.sup_rowptr[s];
      const int ld = (int)(S.sup_rowptr[s + 1] - rp);
      sups[s] = ResSup{(int32_t)dst, f, w, ld, rb, cb, (int32_t)brows.size()};
      store.push_back(ResStoreSup{S.pan_off[s], dst, dst, f, w, ld});
      for (int i = 0; i < ld; ++i) fsup.push_back((uint16_t)s);
      for (int j = 0; j < w; ++j) bsup.push_back((uint16_t)s);
      for (int i = w; i < ld; ++i) {
        up.push_back(Upd{S.sup_rows[rp + i], (int32_t)up.size(), (int32_t)brows.size() - lb});
        brows.push_back(S.sup_rows[rp + i]);
      }
      rb += ld;
      cb += w;
      dst += (int64_t)ld * w;
      fmax = std::max(fmax, w);
      bmax = std::max(bmax, ld);
    }
    std::sort(up.begin(), up.end(), [](const Upd& x, const Upd& y) {
      return x.t != y.t ? x.t < y.t : x.ord < y.ord;
    });
    // target j subtracts the slots tslot[tpp[j-1] .. tpp[j]) (level-local,
    // from 0 for the level's first target)
    for (size_t e = 0; e < up.size(); ++e) {
      tslot.push_back(up[e].slot);
      if (e + 1 == up.size() || up[e + 1].t != up[e].t) {
        tgt.push_back(up[e].t);
        tpp.push_back((int32_t)e + 1);
      }
    }
    uslots = std::max(uslots, (int)up.size());
    at(kResOffFL, l) = lanes(rb, fmax);
    at(kResOffBL, l) = lanes(cb, bmax);
  }
  if (dst > INT32_MAX) return false;
  // tslot entries are level-local; tpp too, but stored after the level's
  // earlier targets: make both absolute within the blob's lists
  {
    int32_t base = 0;
    for (int l = 0; l < nlev; ++l) {
      const int t0 = at(kResOffT, l), t1 = at(kResOffT, l + 1);
      for (int j = t0; j < t1; ++j) tpp[j] += base;
      if (t1 > t0) base = tpp[t1 - 1];
    }
  }
  std::vector<unsigned char> blob;
  auto put = [&](const void* d, size_t bytes) -> int32_t {
    const size_t o = (blob.size() + 15) & ~(size_t)15;
    blob.resize(o + bytes);
    if (bytes) std::memcpy(blob.data() + o, d, bytes);
    return (int32_t)o;
  };
  ResidentPlan P;
  P.o_offs = put(offs.data(), 4 * offs.size());
  P.o_sups = put(sups.data(), sizeof(ResSup) * sups.size());
  P.o_fsup = put(fsup.data(), 2 * fsup.size());
  P.o_bsup = put(bsup.data(), 2 * bsup.size());
  P.o_tgt = put(tgt.data(), 4 * tgt.size());
  P.o_tpp = put(tpp.data(), 4 * tpp.size());
  P.o_tslot = put(tslot.data(), 4 * tslot.size());
  P.o_brows = put(brows.data(), 4 * brows.size());
  blob.resize((blob.size() + 15) & ~(size_t)15);
  P.bytes = (int32_t)blob.size();
  P.nlev = nlev;
  P.uslots = uslots;
  unsigned char* bd = nullptr;
  ResStoreSup* sd = nullptr;
  double *fm = nullptr, *bm = nullptr, *fg = nullptr, *bg = nullptr;
  if (!c->upload(bd, blob.data(), blob.size()) || !c->upload(sd, store.data(), store.size()) ||
      !c->alloc(fm, (size_t)dst) || !c->alloc(bm, (size_t)dst) || !c->alloc(fg, (size_t)dst) ||
      !c->alloc(bg, (size_t)dst))
    return false;
  P.blob = bd;
  c->rplan = P;
  c->rsup = sd;
  c->rM = ResFactor{fm, bm};
  c->rG = ResFactor{fg, bg};
  resident_store(c->fM, sd, (int)store.size(), fm, bm, c->st);
  resident_store(c->fG, sd, (int)store.size(), fg, bg, c->st);
  return cudaStreamSynchronize(c->st) == cudaSuccess;
}

// The single-column level kernels' plan (see K1Plan): per direction and
// level, the level's supernodes sorted by the lanes one output row (column)
// takes, G = 2^lg with 16 G >= its longest dot product (forward: w terms,
// backward: w + r; at most 32 lanes, more trips beyond 512 terms), then by
// that length; and the warps, each 32 / G consecutive rows of one G.
void build_k1_plan(const Symbolic& S, std::vector<K1Sup> (&recs)[2],
                   std::vector<K1Warp> (&warps)[2], std::vector<int32_t> (&off)[2]) {
  const int nlev = (int)S.level_ptr.size() - 1;
  for (int dir = 0; dir < 2; ++dir) {
    recs[dir].clear();
    warps[dir].clear();
    const bool fwd = dir == 0;
    off[dir].assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
      off[dir][l] = (int32_t)warps[dir].size();
      struct Item { int lg, len, cnt; K1Sup d; };
      std::vector<Item> it;
      for (int k = S.level_ptr[l]; k < S.level_ptr[l + 1]; ++k) {
        const int sn = S.level_sups[k];
        K1Sup d{};
        d.f = S.sup_first[sn];
        d.w = S.sup_first[sn + 1] - d.f;
        d.rp = S.sup_rowptr[sn];
        d.ld = (int32_t)(S.sup_rowptr[sn + 1] - d.rp);
        d.po = S.pan_off[sn];
        const int len = fwd ? d.w : d.ld;
        int lg = 0;
        while (lg < 5 && 16 * (1 << lg) < len) ++lg;
        it.push_back(Item{lg, len, fwd ? d.ld : d.w, d});
      }
      std::stable_sort(it.begin(), it.end(), [](const Item& a, const Item& b) {
        return a.lg != b.lg ? a.lg < b.lg : a.len < b.len;
      });
      const int base = (int)recs[dir].size();
      for (const Item& x : it) recs[dir].push_back(x.d);
      for (size_t a = 0; a < it.size();) {
        size_t e = a;
        while (e < it.size() && it[e].lg == it[a].lg) ++e;
        const int per = 32 >> it[a].lg;
        size_t k = a;
        int i0 = 0;
        while (k < e) {
          // the next warp: per rows from (k, i0) on, within this group size
          size_t kk = k;
          int ii = i0, take = 0;
          while (take < per && kk < e) {
            const int use = std::min(it[kk].cnt - ii, per - take);
            take += use;
            ii += use;
            if (ii == it[kk].cnt) {
              ++kk;
              ii = 0;
            }
          }
          warps[dir].push_back(K1Warp{base + (int32_t)k, i0, (int16_t)it[a].lg, (int16_t)take, 0});
          k = kk;
          i0 = ii;
        }
        a = e;
      }
    }
    off[dir][nlev] = (int32_t)warps[dir].size();
  }
}

bool plan_k1(matex_ctx* c) {
  const Symbolic& S = c->S;
  std::vector<K1Sup> recs[2];
  std::vector<K1Warp> warps[2];
  std::vector<int32_t> off[2];
  build_k1_plan(S, recs, warps, off);
  const int nlev = (int)S.level_ptr.size() - 1;
  K1Sup *fs = nullptr, *bs = nullptr;
  K1Warp *fw = nullptr, *bw = nullptr;
  if (!c->upload(fs, recs[0].data(), recs[0].size()) || !c->upload(bs, recs[1].data(), recs[1].size()) ||
      !c->upload(fw, warps[0].data(), warps[0].size()) ||
      !c->upload(bw, warps[1].data(), warps[1].size()))
    return false;
  c->k1_fw_off = off[0];
  c->k1_bw_off = off[1];
  c->k1.nlev = nlev;
  c->k1.nsup = S.nsup;
  c->k1.fsups = fs;
  c->k1.bsups = bs;
  c->k1.fwarps = fw;
  c->k1.bwarps = bw;
  c->k1.fw_off = c->k1_fw_off.data();
  c->k1.bw_off = c->k1_bw_off.data();
  return true;
}

int solve_cols(matex_ctx* c, const DevFactor& F, int ncols);

std::string tune_key(matex_ctx* c);

// opts.single_column 2: the single-column kernels for every solve of one
// column; 0 (with the tuned launch mode): where their solve pair is at least
// 5 % faster than the tuned path's (best of three after a warm-up each),
// cached in MATEX_AUTOTUNE_CACHE like the other tuners' choices.
void autotune_k1(matex_ctx* c) {
  c->k1_use = false;
  if (!plan_k1(c)) return;
  if (c->opts.single_column == 2) {
    c->k1_use = true;
    return;
  }
  const char* cache = std::getenv("MATEX_AUTOTUNE_CACHE");
  const std::string key = "k1:" + tune_key(c);
  if (cache) {
    if (FILE* f = std::fopen(cache, "r")) {
      char line[1024];
      int found = -1;
      while (std::fgets(line, sizeof(line), f)) {
        const std::string l(line);
        if (l.compare(0, key.size() + 1, key + " ") == 0 && l.size() > key.size() + 1)
          found = l[key.size() + 1] == '1' ? 1 : 0;
      }
      std::fclose(f);
      if (found >= 0) {
        c->k1_use = found == 1;
        return;
      }
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(c->Y, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
  auto best_of = [&](bool k1) {
    c->k1_use = k1;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, c->st);
      solve_cols(c, c->fM, 1);
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
    return best;
  };
  const float ref = best_of(false), mine = best_of(true);
  c->k1_use = cudaGetLastError() == cudaSuccess && mine < 0.95f * ref;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cache) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "%s %d\n", key.c_str(), c->k1_use ? 1 : 0);
      std::fclose(f);
    }
  }
}

// Tensor-core products of the wide supernodes (k_sptrsv_tc.cu): their table,
// per level the (supernode, row tile) lists of both directions, and the
// panel slices of both factors.  False when there is no wide supernode or no
// room (at most a quarter of the free memory), and the solves stay FP64.
bool plan_ts(matex_ctx* c) {
  const Symbolic& S = c->S;
  const int nlev = (int)S.level_ptr.size() - 1;
  // the narrow levels launch with the column blocks tuned for the full ones
  for (int l = 0; l < nlev && l < (int)c->levels_n.size(); ++l) {
    c->levels_n[l].kbf = c->levels[l].kbf;
    c->levels_n[l].kbb = c->levels[l].kbb;
  }
  std::vector<int32_t> wid(S.nsup, -1);
  std::vector<TsSup> sups;
  int64_t aF = 0, aB = 0, rF = 0, rB = 0;
  int mtf = 0, mtb = 0;
  for (int32_t s = 0; s < S.nsup; ++s) {
    const int f = S.sup_first[s], w = S.sup_first[s + 1] - f;
    if (w < c->ts_minw) continue;
    const int ld = (int)(S.sup_rowptr[s + 1] - S.sup_rowptr[s]);
    TsSup d{};
    d.pan = S.pan_off[s];
    d.rp = S.sup_rowptr[s];
    d.f = f;
    d.w = w;
    d.ld = ld;
    d.mt_f = ts_row_tiles(ld);
    d.mt_b = ts_row_tiles(w);
    d.a_f = aF;
    aF += (int64_t)ts_a_bytes(ld, w);
    d.a_b = aB;
    aB += (int64_t)ts_a_bytes(w, ld);
    d.rs_f = rF;
    rF += 128LL * d.mt_f;
    d.rs_b = rB;
    rB += 128LL * d.mt_b;
    mtf = std::max(mtf, d.mt_f);
    mtb = std::max(mtb, d.mt_b);
    wid[s] = (int32_t)sups.size();
    sups.push_back(d);
  }
  if (sups.empty()) return false;
  const double need = 2.0 * (double)(aF + aB) + 16.0 * (double)(rF + rB);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (need > 0.25 * (double)free_b) return false;
  std::vector<int32_t> list;
  std::vector<int2> tf, tb;
  std::vector<size_t> lo(nlev + 1), fo(nlev + 1), bo2(nlev + 1);
  for (int l = 0; l < nlev; ++l) {
    lo[l] = list.size();
    fo[l] = tf.size();
    bo2[l] = tb.size();
    for (int k = S.level_ptr[l]; k < S.level_ptr[l + 1]; ++k) {
      const int j = wid[S.level_sups[k]];
      if (j < 0) continue;
      list.push_back(j);
      const int kf = ts_k_slices(sups[j].w), kb = ts_k_slices(sups[j].ld);
      for (int kc = 0; kc < kf; ++kc)
        for (int mt = 0; mt < sups[j].mt_f; ++mt) tf.push_back(make_int2(j, mt | (kc << 16)));
      for (int kc = 0; kc < kb; ++kc)
        for (int mt = 0; mt < sups[j].mt_b; ++mt) tb.push_back(make_int2(j, mt | (kc << 16)));
    }
  }
  lo[nlev] = list.size();
  fo[nlev] = tf.size();
  bo2[nlev] = tb.size();
  int32_t* ld = nullptr;
  int2 *tfd = nullptr, *tbd = nullptr;
  TsSup* sd = nullptr;
  if (!c->upload(sd, sups.data(), sups.size()) || !c->upload(ld, list.data(), list.size()) ||
      !c->upload(tfd, tf.data(), tf.size()) || !c->upload(tbd, tb.data(), tb.size()))
    return false;
  for (int fi = 0; fi < 2; ++fi) {
    if (!c->alloc(c->tsA[fi][0], (size_t)aF / 2) || !c->alloc(c->tsA[fi][1], (size_t)aB / 2) ||
        !c->alloc(c->tsR[fi][0], (size_t)rF) || !c->alloc(c->tsR[fi][1], (size_t)rB))
      return false;
  }
  c->ts_sups = sd;
  c->ts_n = (int)sups.size();
  c->ts_levels.assign(nlev, TsLevel{});
  for (int l = 0; l < nlev; ++l) {
    TsLevel& L = c->ts_levels[l];
    L.nsup = (int32_t)(lo[l + 1] - lo[l]);
    L.list = ld + lo[l];
    L.ntile_f = (int32_t)(fo[l + 1] - fo[l]);
    L.tiles_f = tfd + fo[l];
    L.ntile_b = (int32_t)(bo2[l + 1] - bo2[l]);
    L.tiles_b = tbd + bo2[l];
  }
  for (int fi = 0; fi < 2; ++fi) {
    const DevFactor& F = fi == 0 ? c->fM : c->fG;
    ts_split_panels(F, sd, c->ts_n, mtf, true, c->tsA[fi][0], c->tsR[fi][0], c->st);
    ts_split_panels(F, sd, c->ts_n, mtb, false, c->tsA[fi][1], c->tsR[fi][1], c->st);
  }
  c->ts_mtf = mtf;
  c->ts_mtb = mtb;
  ts_set_limits();
  return cudaStreamSynchronize(c->st) == cudaSuccess;
}

int solve_ts(matex_ctx* c, const DevFactor& F, int fi, int ncols);

// Per column count: whether the level solves put the wide supernodes on the
// tensor cores.  opts.tc_solve 2: always; 0: where the solve pair (level
// launches, best of three) is at least 5 % faster that way, at each column
// count the launch-mode tuner measures (1, 2, 4, ..., the buffer width).
void autotune_ts(matex_ctx* c) {
  c->ts_by_ncols.assign(c->ldy + 1, 0);
  c->ts_min_cols = 0;
  if (c->ts_n == 0) return;
  if (c->opts.tc_solve == 2) {
    std::fill(c->ts_by_ncols.begin(), c->ts_by_ncols.end(), (int8_t)1);
    c->ts_min_cols = 1;
    return;
  }
  std::vector<int> reps;
  for (int r = 1; r <= c->ldy; r *= 2) reps.push_back(r);
  if (reps.back() != c->ldy) reps.push_back(c->ldy);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(c->Y, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
  cudaMemsetAsync(c->Y2, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
  auto best_of = [&](int K, bool ts) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, c->st);
      if (ts) solve_ts(c, c->fM, 0, K);
      else solve_inplace(c->fM, c->levels.data(), (int)c->levels.size(), c->Y, c->Y2, c->ldy, K,
                         c->st, &c->split);
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);  // the first is the warm-up
    }
    return best;
  };
  std::vector<int8_t> use(reps.size(), 0);
  for (size_t b = 0; b < reps.size(); ++b) use[b] = best_of(reps[b], true) < 0.95f * best_of(reps[b], false);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t b = 0; b < reps.size(); ++b) {
    const int lo = reps[b];
    const int hi = b + 1 < reps.size() ? reps[b + 1] - 1 : c->ldy;
    for (int nc = lo; nc <= hi; ++nc) c->ts_by_ncols[nc] = use[b];
    if (use[b] && c->ts_min_cols == 0) c->ts_min_cols = lo;
  }
  cudaGetLastError();
}

// The level-by-level solve pair with the wide supernodes' products on the
// tensor cores (factor index fi: 0 = C + gamma G, 1 = G); returns launches.
int solve_ts(matex_ctx* c, const DevFactor& F, int fi, int ncols) {
  const int nlev = (int)c->levels_n.size();
  int launches = 0;
  int32_t* err = c->d_count + 1;
  for (int l = 0; l < nlev; ++l) {
    solve_level(true, F, c->levels_n[l], c->Y, c->Y2, c->ldy, ncols, c->st, &c->split);
    ts_solve_level(F, c->ts_sups, c->ts_levels[l], true, c->tsA[fi][0], c->tsR[fi][0], c->Y, c->Y2,
                   c->ldy, ncols, err, c->st);
    launches += 3;
  }
  for (int l = nlev - 1; l >= 0; --l) {
    solve_level(false, F, c->levels_n[l], c->Y, c->Y2, c->ldy, ncols, c->st, &c->split);
    ts_solve_level(F, c->ts_sups, c->ts_levels[l], false, c->tsA[fi][1], c->tsR[fi][1], c->Y, c->Y2,
                   c->ldy, ncols, err, c->st);
    launches += 3;
  }
  return launches;
}

int solve_cols(matex_ctx* c, const DevFactor& F, int ncols) {
  if (ncols <= 0) return 0;
  // one column: the single-column level kernels (any factor of this
  // symbolic structure: C + gamma G, G, the trapezoidal one)
  if (ncols == 1 && c->k1_use && F.sup_first == c->fM.sup_first)
    return solve_k1(F, c->k1, c->Y, c->Y2, c->ldy, c->st);
  int mode = c->opts.solve_mode;
  if (mode == 2) mode = c->mode_by_ncols.empty() ? 0 : c->mode_by_ncols[std::min(ncols, c->ldy)];
  const int fi = F.pan_cm == c->fM.pan_cm ? 0 : F.pan_cm == c->fG.pan_cm ? 1 : -1;
  if (mode == 1 && fi >= 0 && c->ts_n > 0 && !c->ts_by_ncols.empty() &&
      c->ts_by_ncols[std::min(ncols, c->ldy)])
    return solve_ts(c, F, fi, ncols);
  if (mode == 1)
    return solve_inplace(F, c->levels.data(), (int)c->levels.size(), c->Y, c->Y2, c->ldy, ncols,
                         c->st, &c->split);
  const int nlev = (int)c->levels.size();
  const int32_t nsup = c->S.nsup;
  PersistSched ps;
  ps.lev = c->plev_d + (size_t)(ncols - 1) * nlev;
  ps.nlev = nlev;
  ps.nf_total = c->pf_total[ncols];
  ps.nb_total = c->pb_total[ncols];
  ps.ticket = c->pcounters;
  int* cnt = reinterpret_cast<int*>(c->pcounters + 1);
  ps.fdone = cnt;
  ps.bdone = cnt + nsup;
  ps.fpend = c->fpend;
  ps.err = c->d_count + 1;
  ps.sup_level = c->sup_level_d;
  ps.nft = c->nft_d;
  ps.nbt = c->nbt_d;
  cudaMemsetAsync(c->pcounters, 0, sizeof(unsigned long long) * (1 + (size_t)nsup), c->st);
  cudaMemcpyAsync(c->fpend, c->fpend_init, sizeof(int) * nsup, cudaMemcpyDeviceToDevice, c->st);
  if (c->inject_wait) bump_counter(c->fpend + (nsup - 1), c->st);
  persistent_solve(F, ps, c->pgrid, c->psmem, c->Y, c->Y2, c->ldy, c->st);
  return 1;
}

RoundCols round_cols(matex_ctx* c, const Round& r) {
  RoundCols rc;
  rc.group = c->rc_group + r.begin;
  rc.vslot = c->rc_vslot + r.begin;
  rc.seg = c->rc_seg + r.begin;
  rc.l0 = c->rc_l0 + r.begin;
  rc.len = c->rc_len + r.begin;
  rc.hfirst = c->rc_hfirst + r.begin;
  rc.lprev = c->rc_lprev + r.begin;
  rc.obeg = c->rc_obeg + r.begin;
  rc.nout = c->rc_nout + r.begin;
  rc.segid = c->rc_segid + r.begin;
  rc.sgroup = c->rc_sgroup + r.begin;
  rc.abort = c->d_count + 2;
  return rc;
}

matex_status read_count(matex_ctx* c, int* out) {
  cudaMemcpyAsync(c->h_count, c->d_count, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "sync");
  *out = c->h_count[0];
  if (c->h_count[1] != 0)
    return fail(c, MATEX_ERR_TIMEOUT, "a bounded wait of the persistent solve expired");
  return MATEX_OK;
}

// Algorithmic work of one batched solve pair with K right-hand sides, from
// the exact fill of L (the explicit zeros of relaxed amalgamation are the
// implementation's choice, not work the method needs): a multiply-add per
// strictly-lower nonzero of L and column in each direction, plus the D^{-1}
// scaling; bytes: L in compressed form (8-byte value and 4-byte row index per
// nonzero, 4-byte column pointers) read once per direction, D^{-1}, and the
// right-hand sides read and written once per direction.
double solve_flops(const matex_ctx* c, int K) {
  return (4.0 * (double)c->S.nnz_L_exact + 2.0 * (double)c->n) * K;
}
double solve_bytes(const matex_ctx* c, int K) {
  return 2.0 * (12.0 * (double)c->S.nnz_L_exact + 4.0 * ((double)c->n + 1.0)) + 8.0 * c->n +
         32.0 * (double)c->n * K;
}

enum { P_SOLVE = 0, P_MOVE = 1, P_GS = 2, P_SMALL = 3, P_RECOMB = 4, P_OTHER = 5 };

// ---- profiling: CUDA events around timed units, summed after the run -------
int prof_begin(matex_ctx* c) {
  if (!c->prof_on) return -1;
  while (c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  const int idx = (int)c->ev_used;
  c->ev_used += 2;
  cudaEventRecord(c->ev_pool[idx], c->st);
  return idx;
}

void prof_end(matex_ctx* c, int e0, int cls, int64_t launches, double flops, double bytes,
              int round = -1) {
  if (e0 < 0) return;
  cudaEventRecord(c->ev_pool[e0 + 1], c->st);
  c->pend.push_back({cls, e0, launches, flops, bytes, round});
}

// after the stream is synchronised: fold the pending units into the profile
void prof_collect(matex_ctx* c, const std::vector<int32_t>& m_seg) {
  for (const auto& p : c->pend) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_pool[p.e0], c->ev_pool[p.e0 + 1]);
    c->prof.ms[p.cls] += ms;
    c->prof.units[p.cls] += 1;
    c->prof.launches[p.cls] += p.launches;
    double fl = p.flops, by = p.bytes;
    if (p.round >= 0 && p.cls == P_SOLVE) {
      // resident round: per column the two G solves and one solve per Arnoldi step
      const Round& r = c->serial ? c->serial_rounds[p.round] : c->rounds[p.round];
      double cols = 0.0;
      for (int q = 0; q < r.K; ++q) cols += 2.0 + m_seg[c->h_segid_all[r.begin + q]];
      fl = cols * solve_flops(c, 1);
      by = cols * solve_bytes(c, 1);
    } else if (p.round >= 0) {
      // recombination: per (node, output, group) m FMAs + the -P term and the sum
      const Round& r = c->serial ? c->serial_rounds[p.round] : c->rounds[p.round];
      const int cover = c->serial ? c->serial_cover[p.round] : c->round_cover[p.round];
      double f = 0.0, vb = 0.0;
      for (int q = 0; q < r.K; ++q) {
        const int64_t sid = c->h_segid_all[r.begin + q];
        const int mq = m_seg[sid];
        f += (double)c->h_nout_all[r.begin + q] * (2.0 * mq + 4.0);
        if (c->h_nout_all[r.begin + q] > 0) vb += mq + 3.0;
      }
      fl = f * (double)c->n;
      by = 8.0 * (double)c->n * (vb + 2.0 * cover);
    }
    c->prof.flops[p.cls] += fl;
    c->prof.bytes[p.cls] += by;
  }
  c->pend.clear();
  c->ev_used = 0;
}


// Sizes of the checkpointed adjoint.  Every segment is recomputed once
// whatever the window, so the window only trades checkpoint memory (fewer
// windows, fewer checkpoints) against window-tape memory (W x Kb segments'
// bases, solve outputs and z'); the block Kb sets how many columns the
// recompute and reverse launches carry.  Chosen: the widest block for which
// some window fits the budget, with the window that needs the least memory.
struct TapePlan {
  int W = 0, Kb = 0;
  double bytes = 0.0;
};
TapePlan plan_tape(const std::vector<Round>& rounds, int64_t n, int G, int Kmax, int n_times,
                   int nrows, double budget, int W_fix, int Kb_fix) {
  const double nd = (double)n;
  auto ck = [&](int W) {
    double s = 0.0;
    for (size_t r = 0; r < rounds.size(); r += (size_t)W) s += rounds[r].K;
    return s * 2.0 * nd * 8.0;
  };
  auto tape = [&](int W, int Kb) {
    const double slots = (double)W * Kb;
    return slots * (kMaxM + 1) * nd * 8.0 + std::max(0.0, slots - G) * kMaxB * nd * 8.0 +
           (double)Kb * kWSlots * nd * 8.0 + 2.0 * Kb * n_times * kCoefLd * 8.0 +
           2.0 * Kb * std::max(nrows, 1) * 8.0;
  };
  const int nr = std::max<int>(1, (int)rounds.size());
  std::vector<int> kbs, ws;
  if (Kb_fix > 0) kbs.push_back(std::min(Kb_fix, std::max(Kmax, 1)));
  else
    for (int k = std::max(Kmax, 1); k >= 1; k = k > 1 ? (k + 1) / 2 : 0) {
      kbs.push_back(k);
      if (k == 1) break;
    }
  if (W_fix > 0) ws.push_back(std::min(W_fix, nr));
  else
    for (int w = 1;; w *= 2) {
      ws.push_back(std::min(w, nr));
      if (w >= nr) break;
    }
  for (int kb : kbs) {
    TapePlan best;
    for (int w : ws) {
      const double b = ck(w) + tape(w, kb);
      if (b <= budget && (best.W == 0 || b < best.bytes)) best = TapePlan{w, kb, b};
    }
    if (best.W) return best;
  }
  return TapePlan{};
}

// Autotuner: for column counts 1, 2, 4, ..., ldy, time the batched solve with
// one persistent launch and with one launch per tree level (CUDA events, best
// of five after a warm-up) and keep level launches unless the persistent one
// is at least 10 % faster, for every column count up to the next measured one.  The choice depends on the factor's tree (how
// many levels, how much work per level) and on the GPU, so it is measured
// rather than fixed.  An optional cache file (MATEX_AUTOTUNE_CACHE) keyed by
// the factor's shape and the device name avoids re-measuring.
std::string tune_key(matex_ctx* c) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, c->device);
  char buf[512];
  std::snprintf(buf, sizeof(buf), "n=%lld;nsup=%d;pan=%lld;lev=%d;ldy=%d;dev=%s", (long long)c->n,
                c->S.nsup, (long long)c->S.pan_off[c->S.nsup], (int)c->levels.size(), c->ldy,
                prop.name);
  for (char* p = buf; *p; ++p)
    if (*p == ' ') *p = '_';
  return buf;
}

// Column block of every level launch, per direction: the tree's levels
// differ (thousands of small supernodes at the bottom, one wide supernode at
// the top), so each level's forward and backward kernel is timed with
// KB = 1, 2, 4 and 8 right-hand sides per thread block at the context's full
// column count (best of three after a warm-up; zero right-hand sides) and
// keeps the fastest.  Blocks whose staging buffer would exceed
// kSolveSmemTune are not tried.  Cached with the launch-mode choice.
void autotune_levels(matex_ctx* c) {
  const std::string key = "kb:" + tune_key(c);
  const char* cache = std::getenv("MATEX_AUTOTUNE_CACHE");
  const int nlev = (int)c->levels.size();
  if (cache) {
    FILE* f = std::fopen(cache, "r");
    if (f) {
      char line[8192];
      bool found = false;
      while (!found && std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        if (l.compare(0, key.size() + 1, key + " ") != 0) continue;
        std::vector<int> v;
        for (size_t i = key.size() + 1; i < l.size(); ++i)
          if (l[i] >= '1' && l[i] <= '8') v.push_back(l[i] - '0');
        if ((int)v.size() == 2 * nlev) {
          for (int k = 0; k < nlev; ++k) {
            c->levels[k].kbf = v[2 * k];
            c->levels[k].kbb = v[2 * k + 1];
          }
          found = true;
        }
      }
      std::fclose(f);
      if (found) return;
    }
  }
  cudaMemsetAsync(c->Y, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
  cudaMemsetAsync(c->Y2, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
  c->level_tune_ms.assign(2 * nlev, -1.f);
  for (int l = 0; l < nlev; ++l) {
    LevelPlan& L = c->levels[l];
    for (int dir = 0; dir < 2; ++dir) {
      const bool fwd = dir == 0;
      const int ext = fwd ? L.max_w : L.max_wr;
      int best_kb = fwd ? L.kbf : L.kbb;
      float best = 1e30f;
      for (int kb = 1; kb <= kMaxColBlock; kb *= 2) {
        if ((size_t)ext * kb * sizeof(double) > (size_t)kSolveSmemTune) break;
        const float ms = time_level(fwd, c->fM, L, kb, c->Y, c->Y2, c->ldy, c->ldy, c->st,
                                    &c->split, 3);
        if (ms > 0.f && ms < best) {
          best = ms;
          best_kb = kb;
        }
      }
      (fwd ? L.kbf : L.kbb) = best_kb;
      c->level_tune_ms[2 * l + dir] = best < 1e29f ? best : -1.f;
    }
  }
  if (cache) {
    FILE* f = std::fopen(cache, "a");
    if (f) {
      std::fprintf(f, "%s ", key.c_str());
      for (int l = 0; l < nlev; ++l) std::fprintf(f, "%d%d", c->levels[l].kbf, c->levels[l].kbb);
      std::fprintf(f, "\n");
      std::fclose(f);
    }
  }
}

void autotune_solve(matex_ctx* c) {
  c->mode_by_ncols.assign(c->ldy + 1, 0);
  c->tune_reps.clear();
  c->tune_modes.clear();
  c->tune_ms.clear();
  for (int r = 1; r <= c->ldy; r *= 2) c->tune_reps.push_back(r);
  if (c->tune_reps.back() != c->ldy) c->tune_reps.push_back(c->ldy);
  const char* cache = std::getenv("MATEX_AUTOTUNE_CACHE");
  const std::string key = tune_key(c);
  bool found = false;
  if (cache) {
    FILE* f = std::fopen(cache, "r");
    if (f) {
      char line[1024];
      while (std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        if (l.compare(0, key.size() + 1, key + " ") != 0) continue;
        std::vector<int32_t> modes;
        for (size_t i = key.size() + 1; i < l.size(); ++i)
          if (l[i] == '0' || l[i] == '1') modes.push_back(l[i] - '0');
        if (modes.size() == c->tune_reps.size()) {
          c->tune_modes = modes;
          found = true;
        }
      }
      std::fclose(f);
    }
  }
  if (!found) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(c->Y, 0, sizeof(double) * (size_t)c->n * c->ldy, c->st);
    const int saved = c->opts.solve_mode;
    for (int r : c->tune_reps) {
      float best[2] = {1e30f, 1e30f};
      for (int mode = 0; mode < 2; ++mode) {
        c->opts.solve_mode = mode;
        solve_cols(c, c->fM, r);
        for (int rep = 0; rep < 5; ++rep) {
          cudaEventRecord(e0, c->st);
          solve_cols(c, c->fM, r);
          cudaEventRecord(e1, c->st);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          best[mode] = std::min(best[mode], ms);
        }
      }
      // one persistent launch only when clearly faster: the two modes' times
      // differ by a few percent from process to process, and level launches
      // are the better-tested path (and the one the column-block tuner tuned)
      c->tune_modes.push_back(best[0] < 0.9f * best[1] ? 0 : 1);
      c->tune_ms.push_back(best[0]);
      c->tune_ms.push_back(best[1]);
    }
    c->opts.solve_mode = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache) {
      FILE* f = std::fopen(cache, "a");
      if (f) {
        std::fprintf(f, "%s ", key.c_str());
        for (int32_t m : c->tune_modes) std::fprintf(f, "%d", m);
        std::fprintf(f, "\n");
        std::fclose(f);
      }
    }
  }
  for (size_t b = 0; b < c->tune_reps.size(); ++b) {
    const int lo = c->tune_reps[b];
    const int hi = b + 1 < c->tune_reps.size() ? c->tune_reps[b + 1] - 1 : c->ldy;
    for (int nc = lo; nc <= hi; ++nc) c->mode_by_ncols[nc] = (int8_t)c->tune_modes[b];
  }
}

// G in CSR in the factor's permuted order on the device (the trapezoidal
// baseline and the standard Krylov space apply G itself).
bool ensure_g_csr(matex_ctx* c) {
  if (c->trG_rowptr) return true;
  const int64_t n = c->n;
  const Symbolic& S = c->S;
  std::vector<int64_t> rp(n + 1, 0);
  for (int64_t k = 0; k < n; ++k) {
    const int32_t o = S.perm[k];
    rp[k + 1] = rp[k] + (c->g_rowptr_h[o + 1] - c->g_rowptr_h[o]);
  }
  std::vector<int32_t> col(rp[n]);
  std::vector<double> val(rp[n]);
  for (int64_t k = 0; k < n; ++k) {
    const int32_t o = S.perm[k];
    int64_t d = rp[k];
    for (int64_t e = c->g_rowptr_h[o]; e < c->g_rowptr_h[o + 1]; ++e, ++d) {
      col[d] = S.iperm[c->g_col_h[e]];
      val[d] = c->g_val_h[e];
    }
  }
  int64_t* r = nullptr;
  int32_t* cl = nullptr;
  double* v = nullptr;
  if (!c->upload(r, rp.data(), rp.size()) || !c->upload(cl, col.data(), col.size()) ||
      !c->upload(v, val.data(), val.size()))
    return false;
  c->trG_rowptr = r;
  c->trG_col = cl;
  c->trG_val = v;
  return true;
}

// One pass of the run (everything up to the output permutation) on c->st.
// Plain (capture = false): the host reads every active-column count from the
// device and appends it to kit_trace.  Recording (capture = true): the stream
// is being captured into a CUDA graph; each count is taken from kit_trace and
// followed by a guard kernel that raises the divergence flag (and keeps every
// index in range) if the device count differs when the graph is replayed.
matex_status run_pass(matex_ctx* c, bool capture, PassCounts& pc) {
  cudaStream_t st = c->st;
  const int64_t n = c->n;
  const double nd = (double)n;
  const int64_t vstride = (int64_t)kMaxB * n;
  int launches = 0, sweepsM = 0, sweepsG = 0;
  int64_t solve_cols_total = 0;
  int e;
  size_t tpos = 0;
  auto count = [&](int* out, int32_t* iter_now, const int32_t* vslot) -> matex_status {
    if (!capture) {
      const matex_status rs = read_count(c, out);
      if (rs == MATEX_OK) c->kit_trace.push_back(*out);
      return rs;
    }
    if (tpos >= c->kit_trace.size()) return fail(c, MATEX_ERR_STATE, "count trace too short");
    *out = c->kit_trace[tpos++];
    expect_count(c->d_count, *out, iter_now, c->iter_grp, vslot, c->d_count + 2, st);
    launches++;
    return MATEX_OK;
  };
  cudaMemsetAsync(c->d_count, 0, 4 * sizeof(int32_t), st);
  auto solve = [&](const DevFactor& F, int K) {
    e = prof_begin(c);
    int l = 1;
    // resident rounds: the DC and initial-state solves by the same one-CTA
    // substitution (no atomics anywhere in such a run: reproducible)
    if (c->resident)
      resident_solve(&F == &c->fM ? c->rM : c->rG, c->rplan, c->Y, c->Y, n, K, c->ldy, 1, nullptr, st);
    else l = solve_cols(c, F, K);
    prof_end(c, e, P_SOLVE, l, solve_flops(c, K), solve_bytes(c, K));
    launches += l;
    solve_cols_total += K;
  };
  auto moved = [&](int e0, int nl, int K, bool scaled) {
    prof_end(c, e0, P_MOVE, nl, scaled ? nd * K : 0.0, 16.0 * nd * K * nl);
    launches += nl;
  };
  // constant part: x_dc = G^{-1} dc_inject
  if (c->opts.include_dc && c->dc_perm) {
    e = prof_begin(c);
    gather_cols(c->Y, c->ldy, 1, c->dc_perm, 0, nullptr, nullptr, nullptr, n, st);
    moved(e, 1, 1, false);
    solve(c->fG, 1);
    sweepsG++;
    e = prof_begin(c);
    scatter_cols(c->Y, c->ldy, 1, c->xdc, 0, nullptr, nullptr, n, st);
    moved(e, 1, 1, false);
    e = prof_begin(c);
    fill_rows(c->Xp, c->xdc, n, c->n_times, st);
    prof_end(c, e, P_OTHER, 1, 0.0, 8.0 * nd * (c->n_times + 1));
    launches++;
  } else {
    e = prof_begin(c);
    fill_rows(c->Xp, nullptr, n, c->n_times, st);
    prof_end(c, e, P_OTHER, 1, 0.0, 8.0 * nd * c->n_times);
    launches++;
  }
  // per-run state starts at zero: x, z, z' of every group, the segment records
  {
    const size_t gb = sizeof(double) * (size_t)c->g_slots * (size_t)n;
    cudaMemsetAsync(c->Xb, 0, gb, st);
    cudaMemsetAsync(c->Zb, 0, gb, st);
    cudaMemsetAsync(c->Zpb, 0, gb, st);
    cudaMemsetAsync(c->m_rec, 0, sizeof(int32_t) * std::max<int64_t>(1, c->n_segments), st);
    cudaMemsetAsync(c->st_rec, 0, sizeof(int32_t) * std::max<int64_t>(1, c->n_segments), st);
  }
  matex_status s = MATEX_OK;
  const std::vector<Round>& rounds = c->serial ? c->serial_rounds : c->rounds;
  const size_t nbatch = c->serial ? 1 : c->batches.size();
  for (size_t bi = 0; bi < nbatch; ++bi) {
  const int r0 = c->serial ? 0 : c->batches[bi].r0;
  const int r1 = c->serial ? (int)rounds.size() : c->batches[bi].r1;
  const int i0 = c->serial ? 0 : c->batches[bi].i0;
  const int ng = c->serial ? (int)c->init_groups.size() : c->batches[bi].ni;
  if (bi > 0) {
    // the batch's groups take over the previous batch's state slots
    const size_t gb = sizeof(double) * (size_t)c->g_slots * (size_t)n;
    cudaMemsetAsync(c->Xb, 0, gb, st);
    cudaMemsetAsync(c->Zb, 0, gb, st);
    cudaMemsetAsync(c->Zpb, 0, gb, st);
  }
  // each group's own DC state at t = 0 (Alg. 2's local initial solution); groups with
  // zero input at t = 0 start from x = 0
  for (int g0 = 0; g0 < ng; g0 += c->ldy) {
    const int K = std::min(c->ldy, ng - g0);
    e = prof_begin(c);
    build_initial_rhs(c->Y, c->ldy, K, c->src, c->init_groups_d + i0 + g0, n, st);
    prof_end(c, e, P_OTHER, 2, 0.0, 8.0 * nd * c->ldy);
    launches += 2;
    solve(c->fG, K);
    sweepsG++;
    e = prof_begin(c);
    scatter_cols(c->Y, c->ldy, K, c->Xb, n, c->init_slots_d + i0 + g0, nullptr, n, st);
    moved(e, 1, K, false);
    e = prof_begin(c);
    add_row_sum(c->Xp, c->Y, c->ldy, K, n, st);
    prof_end(c, e, P_OTHER, 1, nd * K, 8.0 * nd * (K + 2));
    launches++;
  }
  s = cuda_check(c, "initial states");
  if (s != MATEX_OK) return s;
  auto res_args = [&](const Round& r) {
    ResidentArgs ra{};
    ra.F1 = c->opts.krylov == 1 ? c->rG : c->rM;
    ra.FG = c->rG;
    ra.plan = c->rplan;
    ra.cperm = c->c_perm;
    ra.src = c->src;
    ra.rc = round_cols(c, r);
    ra.n = n;
    if (c->pre_zp) {
      ra.zpre = c->pre_zp + (int64_t)r.begin * n;
      ra.wpre = c->pre_w + (int64_t)r.begin * n;
    }
    return ra;
  };
  if (c->resident && c->pre_zp && bi == 0) {
    // the input solves of every column record (sources only, no state): one
    // launch, one CTA per record, instead of two solves in each round kernel
    Round all;
    all.begin = 0;
    all.K = (int32_t)c->n_records;
    e = prof_begin(c);
    resident_inputs(res_args(all), all.K, st);
    prof_end(c, e, P_SOLVE, 1, 2.0 * solve_flops(c, 1) * all.K, 2.0 * solve_bytes(c, 1) * all.K);
    launches++;
    sweepsG += 2;
    solve_cols_total += 2 * c->n_records;
    if ((s = cuda_check(c, "input solves")) != MATEX_OK) return s;
  }
  for (size_t ri = (size_t)r0; ri < (size_t)r1; ++ri) {
    const Round& r = rounds[ri];
    const int K = r.K;
    RoundCols rc = round_cols(c, r);
    if (c->resident) {
      // every column's whole segment in one launch (one CTA each), then the
      // recombination of the round's outputs
      ResidentArgs ra = res_args(r);
      ra.Vb = c->Vb;
      ra.vstride = vstride;
      ra.X = c->Xb;
      ra.Z = c->Zb;
      ra.Zp = c->Zpb;
      ra.W = c->Wb;
      ra.ss = c->ss;
      ra.coef = c->coef;
      ra.ldo = c->n_times;
      ra.yend = c->yend;
      ra.m_rec = c->m_rec;
      ra.st_rec = c->st_rec;
      ra.replay = c->replay_d;
      ra.gamma = c->gamma;
      ra.tol = c->tol;
      ra.dt_out = c->dt_out;
      ra.m_max = c->m_max;
      e = prof_begin(c);
      resident_round(ra, K, st);
      prof_end(c, e, P_SOLVE, 1, 0.0, 0.0, (int)ri);
      e = prof_begin(c);
      recombine(c->Xp, n, c->n_times, c->Vb, vstride, c->Zb, c->Zpb, c->Wb, n, rc, c->ss.m, c->coef,
                c->n_times, K, r.obeg_min, r.oend_max, c->dt_out, st, nullptr);
      prof_end(c, e, P_RECOMB, 1, 0.0, 0.0, (int)ri);
      launches += 2;
      if (!c->pre_zp) {
        sweepsG += 2;
        solve_cols_total += 2 * (int64_t)K;
      }
      if ((s = cuda_check(c, "round")) != MATEX_OK) return s;
      continue;
    }
    // z = G^{-1} B u(l_j) carried forward (u is continuous and linear on every
    // segment: z_j = z_{j-1} + L_{j-1} z'_{j-1}, z_0 = x(0)); then
    // z' = G^{-1} B s_j and w = G^{-1} C z'   (Eq. 5/6)
    e = prof_begin(c);
    advance_z(c->Zb, c->Zpb, c->Xb, n, rc, K, n, st);
    if (c->opts.tape == 2 && !c->serial && ri % (size_t)c->tape_W == 0) {
      // adjoint checkpoint: x and z of every column at the start of the window
      checkpoint_states(c->CK + c->ck_base[ri / c->tape_W] * 2 * n, c->Xb, c->Zb, rc.group, K, n,
                        false, st);
      launches++;
    }
    build_input_rhs(c->Y, c->ldy, K, rc, c->src, n, st);
    prof_end(c, e, P_OTHER, 3, 2.0 * nd * K, 24.0 * nd * K + 8.0 * nd * c->ldy);
    launches += 3;
    solve(c->fG, K);
    e = prof_begin(c);
    scatter_cols(c->Y, c->ldy, K, c->Zpb, n, rc.group, nullptr, n, st);
    if (c->opts.tape == 1) scatter_cols(c->Y, c->ldy, K, c->TZp, n, rc.vslot, nullptr, n, st);
    gather_cols(c->Y, c->ldy, K, c->Zpb, n, rc.group, c->c_perm, nullptr, n, st);
    moved(e, 2, K, true);
    solve(c->fG, K);
    e = prof_begin(c);
    scatter_cols(c->Y, c->ldy, K, c->Wb, n, rc.group, nullptr, n, st);
    moved(e, 1, K, false);
    sweepsG += 2;
    // start vector v = x + F, beta = ||v||
    e = prof_begin(c);
    krylov_start(c->Vb, vstride, c->Xb, c->Zb, c->Wb, n, rc.group, rc.vslot, K, n, c->partials,
                 c->nchunks, st);
    prof_end(c, e, P_OTHER, 1, 4.0 * nd * K, 32.0 * nd * K);
    e = prof_begin(c);
    start_finish(c->partials, c->nchunks, K, c->ss, rc.vslot, c->iterA, c->iter_grp, c->d_count, st);
    prof_end(c, e, P_SMALL, 1, 0.0, 0.0);
    launches += 2;
    int kit = 0;
    int32_t* iter = c->iterA;
    int32_t* iter_next = c->iterB;
    if ((s = count(&kit, iter, rc.vslot)) != MATEX_OK) return s;
    if (kit > 0) {
      e = prof_begin(c);
      basis_scale(c->Vb, vstride, rc.vslot, iter, kit, 0, c->ss.scale, n, st);
      prof_end(c, e, P_GS, 1, nd * kit, 16.0 * nd * kit);
      launches++;
    }
    int kdim = 0;  // basis vectors of the round: each Arnoldi step adds one per active column
    for (int j = 0; j < c->m_max && kit > 0; ++j) {
      kdim += kit;
      if (c->opts.krylov == 2) {
        // standard space (MEXP): w = A v_j = -C^{-1} G v_j, no solve
        e = prof_begin(c);
        krylov_apply_A(c->Vb, vstride, c->iter_grp, kit, j, j + 1, c->trG_rowptr, c->trG_col,
                       c->trG_val, c->c_perm, n, st);
        prof_end(c, e, P_SOLVE, 1, 2.0 * (double)c->g_col_h.size() * kit,
                 (12.0 * (double)c->g_col_h.size() + 24.0 * nd) * kit);
        launches++;
      } else {
        // w = X1^{-1} C v_j   (Alg. 1 with X2 = C; X1 = C + gamma G, or G for the
        // inverted space)
        e = prof_begin(c);
        gather_cols(c->Y, c->ldy, kit, c->Vb + (int64_t)j * n, vstride, c->iter_grp, c->c_perm,
                    nullptr, n, st);
        moved(e, 1, kit, true);
        solve(c->opts.krylov == 1 ? c->fG : c->fM, kit);
        e = prof_begin(c);
        scatter_cols(c->Y, c->ldy, kit, c->Vb + (int64_t)(j + 1) * n, vstride, c->iter_grp, nullptr,
                     n, st);
        if (c->opts.tape == 1)  // keep a_k = (C + gamma G)^{-1} C q_k for the adjoint
          scatter_cols(c->Y, c->ldy, kit, c->TA + (int64_t)j * n, (int64_t)kMaxM * n, c->iter_grp,
                       nullptr, n, st);
        moved(e, 1, kit, false);
      }
      sweepsM++;
      // two classical Gram-Schmidt passes, then the norm and the normalisation
      e = prof_begin(c);
      for (int pass = 0; pass < 2; ++pass) {
        basis_dots(c->Vb, vstride, rc.vslot, iter, kit, 0, j + 1, j + 1, n, c->partials,
                   c->nchunks, st);
        reduce_dots(c->partials, c->nchunks, kit, j + 1, iter, c->ss, j, pass, st);
        basis_update(c->Vb, vstride, rc.vslot, iter, kit, j + 1, j + 1, c->ss.hbuf, n, st);
      }
      basis_dots(c->Vb, vstride, rc.vslot, iter, kit, j + 1, 1, j + 1, n, c->partials, c->nchunks,
                 st);
      reduce_dots(c->partials, c->nchunks, kit, 1, iter, c->ss, j, 2, st);
      basis_scale(c->Vb, vstride, rc.vslot, iter, kit, j + 1, c->ss.scale, n, st);
      prof_end(c, e, P_GS, 9, (8.0 * j + 11.0) * nd * kit, (4.0 * j + 13.0) * 8.0 * nd * kit);
      e = prof_begin(c);
      residual_check(c->ss, rc, kit, j, c->gamma, c->tol, c->m_max, c->replay_d, iter, iter_next,
                     c->iter_grp, c->d_count, st);
      prof_end(c, e, P_SMALL, 2, 0.0, 0.0);
      launches += 11;
      std::swap(iter, iter_next);
      if ((s = count(&kit, iter, rc.vslot)) != MATEX_OK) return s;
    }
    if (c->opts.tape == 1) tape_small(c->ss, rc, K, c->THt, c->Tbeta, st);
    e = prof_begin(c);
    const double teps = c->opts.tail_eps;
    if (teps > 0.0) {
      e = prof_begin(c);
      p_bound(c->Zb, c->Zpb, c->Wb, n, rc, K, n, c->pbound, st);
      prof_end(c, e, P_OTHER, 1, 3.0 * nd * K, 24.0 * nd * K);
      launches++;
    }
    e = prof_begin(c);
    output_coefficients(c->ss, rc, K, c->gamma, c->dt_out, c->coef, c->n_times, c->yend, st,
                        teps, teps > 0.0 ? c->pbound : nullptr, c->tcut);
    prof_end(c, e, P_SMALL, 1, 0.0, 0.0);
    e = prof_begin(c);
    int rl = 1;
    if (c->tc.kdim_cap && teps == 0.0 && kdim >= kTcMinKdim && kdim <= c->tc.kdim_cap &&
        r.cover >= kTcMinCover) {
      // V y on the tensor cores (a dense product over the round's output
      // range, worth it when the columns hold most of that range), then the
      // -P terms alone in one sweep over the outputs
      rl += recombine_tc(c->Xp, n, c->Vb, vstride, rc, c->ss.m, c->coef, c->n_times, K, kdim,
                         r.obeg_min, r.oend_max, c->tc, st);
      pc.tc_rounds++;
      recombine_p(c->Xp, n, c->Zb, c->Zpb, c->Wb, n, rc, c->ev_o_d + r.ev_begin,
                  c->ev_q_d + r.ev_begin, r.nev, r.obeg_min, r.oend_max, c->dt_out, st);
    } else {
      recombine(c->Xp, n, c->n_times, c->Vb, vstride, c->Zb, c->Zpb, c->Wb, n, rc, c->ss.m, c->coef,
                c->n_times, K, r.obeg_min, r.oend_max, c->dt_out, st,
                teps > 0.0 ? c->tcut : nullptr);
    }
    prof_end(c, e, P_RECOMB, rl, 0.0, 0.0, (int)ri);
    launches += rl - 1;
    e = prof_begin(c);
    next_state(c->Xb, c->Vb, vstride, c->Zb, c->Zpb, c->Wb, n, rc, c->ss.m, c->yend, K, n, st);
    record_segments(c->ss, rc, K, c->m_rec, c->st_rec, st);
    prof_end(c, e, P_OTHER, 2, 0.0, 0.0);
    launches += 4;
    if ((s = cuda_check(c, "round")) != MATEX_OK) return s;
  }
  }
  pc.launches = launches;
  pc.sweepsM = sweepsM;
  pc.sweepsG = sweepsG;
  pc.solve_cols = solve_cols_total;
  return MATEX_OK;
}

void drop_graph(matex_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

// Record the run as a CUDA graph from the count trace of the plain run that
// just finished.  Capture needs a stream other than the legacy default one, so
// the pass is issued on the context's private capture stream.  On any failure
// the context keeps running plainly.
void capture_graph(matex_ctx* c) {
  drop_graph(c);
  const double t = now_ms();
  if (!c->gst && cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->gst = nullptr;
    return;
  }
  cudaGetLastError();
  cudaStream_t user = c->st;
  c->st = c->gst;
  cudaGraph_t g = nullptr;
  PassCounts pc;
  bool ok = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  const std::string saved_err = c->err;
  const matex_status s = ok ? run_pass(c, true, pc) : MATEX_ERR_CUDA;
  if (ok) ok = cudaStreamEndCapture(c->gst, &g) == cudaSuccess && s == MATEX_OK && g != nullptr;
  c->st = user;
  c->err = saved_err;
  if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
  if (ok) {
    c->graph = g;
    c->graph_counts = pc;
    c->graph_gen++;
  } else {
    if (g) cudaGraphDestroy(g);
    c->gexec = nullptr;
    cudaGetLastError();
  }
  c->graph_ms = now_ms() - t;
}

bool graph_allowed(const matex_ctx* c) { return c->opts.graph && !c->prof_on && !c->inject_wait; }

// Statistics of the run that just completed (stream synchronised).
matex_status finish_run(matex_ctx* c, const PassCounts& pc, double t0, bool replayed,
                        matex_stats* stats) {
  std::vector<int32_t> m(c->n_segments), stt(c->n_segments);
  if (c->n_segments) {
    if (cudaMemcpy(m.data(), c->m_rec, sizeof(int32_t) * c->n_segments, cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(stt.data(), c->st_rec, sizeof(int32_t) * c->n_segments, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
      return cuda_check(c, "run records");
  }
  matex_stats& o = c->last;
  o = c->setup_stats;
  o.run_ms = now_ms() - t0;
  o.n_segments = (int32_t)c->n_segments;
  o.krylov_segments = o.sum_m = o.max_m = o.nonconv = o.breakdowns = 0;
  for (int64_t i = 0; i < c->n_segments; ++i) {
    if (m[i] > 0) o.krylov_segments++;
    o.sum_m += m[i];
    o.max_m = std::max(o.max_m, m[i]);
    if (stt[i] == 3) o.nonconv++;
    if (stt[i] == 2) o.breakdowns++;
  }
  o.sweeps_M = pc.sweepsM;
  o.tc_rounds = pc.tc_rounds;
  o.sweeps_G = pc.sweepsG;
  o.solve_columns = pc.solve_cols;
  if (c->resident) {
    // the Arnoldi steps were taken on the device: one solve column each
    const std::vector<Round>& rr = c->serial ? c->serial_rounds : c->rounds;
    int64_t sm = 0;
    int32_t sweeps = 0;
    for (const Round& r : rr) {
      int mx = 0;
      for (int q = 0; q < r.K; ++q) {
        const int mq = m[c->h_segid_all[r.begin + q]];
        sm += mq;
        mx = std::max(mx, mq);
      }
      sweeps += mx;
    }
    o.solve_columns += sm;
    o.sweeps_M = sweeps;
  }
  o.kernel_launches = pc.launches + 1;  // + the output permutation
  o.rounds = (int32_t)(c->serial ? c->serial_rounds.size() : c->rounds.size());
  o.graph_replay = replayed ? 1 : 0;
  o.graph_capture_ms = c->graph_ms;
  c->taped = c->opts.tape && !c->serial;
  if (!replayed) prof_collect(c, m);
  if (stats) *stats = o;
  if (c->opts.strict && o.nonconv > 0)
    return fail(c, MATEX_ERR_NOCONV, "some segments reached m_max above tol");
  return MATEX_OK;
}

// Device flags after a replay: 0 = consistent, 1 = counts diverged; an
// expired bounded wait is an error.
matex_status replay_flags(matex_ctx* c, bool* diverged) {
  cudaMemcpyAsync(c->h_count, c->d_count, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "replay sync");
  if (c->h_count[1] != 0)
    return fail(c, MATEX_ERR_TIMEOUT, "a bounded wait of the persistent solve expired");
  *diverged = c->h_count[2] != 0;
  return MATEX_OK;
}

matex_status run_device(matex_ctx* c, double* x_out, matex_stats* stats) {
  const double t0 = now_ms();
  matex_status s;
  if (graph_allowed(c) && c->gexec) {
    if (cudaGraphLaunch(c->gexec, c->st) != cudaSuccess) return cuda_check(c, "graph launch");
    permute_out(x_out, c->Xp, c->out_map, c->nrows_out, c->n, c->n_times, c->st);
    if ((s = cuda_check(c, "graph run")) != MATEX_OK) return s;
    bool diverged = false;
    if ((s = replay_flags(c, &diverged)) != MATEX_OK) return s;
    if (!diverged) return finish_run(c, c->graph_counts, t0, true, stats);
    drop_graph(c);  // the counts changed: run plainly and record again
  }
  c->kit_trace.clear();
  PassCounts pc;
  if ((s = run_pass(c, false, pc)) != MATEX_OK) return s;
  const int e = prof_begin(c);
  permute_out(x_out, c->Xp, c->out_map, c->nrows_out, c->n, c->n_times, c->st);
  prof_end(c, e, P_OTHER, 1, 0.0, 16.0 * (double)c->nrows_out * c->n_times);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "run sync");
  if ((s = cuda_check(c, "run")) != MATEX_OK) return s;
  {
    int tmp = 0;
    if ((s = read_count(c, &tmp)) != MATEX_OK) return s;
  }
  if (graph_allowed(c)) capture_graph(c);
  return finish_run(c, pc, t0, false, stats);
}

// Reverse of the columns [qa, qa + K) of round r, given their tape entries
// (slots rec, device) and the run's Krylov dimension per column record
// (mrec, host; c->mrec_d on the device).  The groups' carried adjoints (xbar
// into the previous segment, zbar, dL/dc) are per group, so any subset of a
// round's columns can be reversed on its own once the later rounds of the
// same groups are.
matex_status reverse_round(matex_ctx* c, const Round& r, int qa, int K, const int32_t* rec,
                           const std::vector<int32_t>& mrec, const double* xbar, double* damp,
                           const SourceTable& base) {
  if (K <= 0) return MATEX_OK;
  cudaStream_t st = c->st;
  const int64_t n = c->n;
  const int nrows = c->nrows_out;
  const int64_t vstride = (int64_t)kMaxB * n;
  const int b0 = r.begin + qa;
  AdjWork aw{c->AW, (int64_t)kWSlots * n, c->XBg, c->CARRYg, c->CBg};
  AdjRound ar;
  ar.rec = rec;
  ar.group = c->rc_group + b0;
  ar.m = c->mrec_d + b0;
  ar.obeg = c->rc_obeg + b0;
  ar.nout = c->rc_nout + b0;
  ar.seg = c->rc_seg + b0;
  ar.l0 = c->rc_l0 + b0;
  ar.len = c->rc_len + b0;
  ar.hfirst = c->rc_hfirst + b0;
  ar.V = c->Vb;
  ar.vstride = vstride;
  ar.A = c->TA;
  ar.astride = (int64_t)kMaxM * n;
  ar.Zp = c->TZp;
  ar.Ht = c->THt;
  ar.beta = c->Tbeta;
  ar.n = n;
  ar.dt = c->dt_out;
  int mmax = 0;
  for (int q = 0; q < K; ++q) mmax = std::max(mmax, mrec[b0 + q]);
  // active column lists for k = 0..mmax-1, uploaded once
  std::vector<int32_t> act;
  std::vector<int> aoff(mmax + 1, 0);
  for (int k = 0; k < mmax; ++k) {
    aoff[k] = (int)act.size();
    for (int q = 0; q < K; ++q)
      if (mrec[b0 + q] > k) act.push_back(q);
  }
  aoff[mmax] = (int)act.size();
  if (!act.empty())
    cudaMemcpyAsync(c->act_d, act.data(), sizeof(int32_t) * act.size(), cudaMemcpyHostToDevice, st);
  // output adjoints and the small dense reverse
  if (mmax > 0) {
    AdjDots d{c->XBg, n, ar.group, 0, c->Vb, vstride, ar.rec, 0, nullptr};
    adj_dots(d, K, mmax, n, c->partials, c->nchunks, c->YBL, st);
  }
  adj_obs(ar, K, xbar, c->out_map, nrows, c->YBO, c->n_times, c->S1, c->S2, st);
  adj_small(ar, K, c->gamma, c->YBO, c->n_times, c->YBL, c->YOUT, c->YL, c->HTB, c->BETAB, st);
  adj_build(ar, aw, K, c->YL, xbar, c->out_map, nrows, c->YOUT, c->n_times, c->S1, c->S2, st);
  // reverse Arnoldi steps
  for (int k = mmax - 1; k >= 0; --k) {
    const int Ka = aoff[k + 1] - aoff[k];
    const int32_t* ak = c->act_d + aoff[k];
    AdjDots d1{c->AW, (int64_t)kWSlots * n, c->iota_d, k + 1, c->Vb, vstride, ar.rec, k + 1, ak};
    adj_dots(d1, Ka, 1, n, c->partials, c->nchunks, c->D1, st);
    adj_rbar(ar, aw, ak, Ka, k, c->D1, c->HTB, st);
    AdjDots dh{c->AW, (int64_t)kWSlots * n, c->iota_d, kWR, c->Vb, vstride, ar.rec, 0, ak};
    adj_dots(dh, Ka, k + 1, n, c->partials, c->nchunks, c->HD, st);
    adj_abar(ar, aw, ak, Ka, k, c->HD, c->HTB, st);
    gather_cols(c->Y, c->ldy, Ka, c->AW + (int64_t)kWA * n, (int64_t)kWSlots * n, ak, nullptr,
                nullptr, n, st);
    solve_cols(c, c->fM, Ka);
    adj_after_m(ar, aw, ak, Ka, k, c->Y, c->ldy, c->c_perm, st);
  }
  {
    AdjDots d0{c->AW, (int64_t)kWSlots * n, c->iota_d, 0, c->Vb, vstride, ar.rec, 0, nullptr};
    if (mmax > 0) adj_dots(d0, K, 1, n, c->partials, c->nchunks, c->D0, st);
  }
  adj_vbar(ar, aw, K, c->D0, c->BETAB, st);
  // w = G^{-1}(c z'), then z' = G^{-1} B s
  gather_cols(c->Y, c->ldy, K, c->AW + (int64_t)kWW * n, (int64_t)kWSlots * n, nullptr, nullptr,
              nullptr, n, st);
  solve_cols(c, c->fG, K);
  adj_after_w(ar, aw, K, c->Y, c->ldy, c->c_perm, st);
  gather_cols(c->Y, c->ldy, K, c->AW + (int64_t)kWZp * n, (int64_t)kWSlots * n, nullptr, nullptr,
              nullptr, n, st);
  solve_cols(c, c->fG, K);
  adj_sources(ar, K, base, c->Y, c->ldy, damp, st);
  return cuda_check(c, "grad round");
}

// Forward of rounds [r0, r1) for the columns [qa[i], qb[i]) of round r0 + i
// (the block's groups) from the checkpoint of window w, keeping each
// segment's basis, solve outputs, z', Hessenberg and norm in window-tape slot
// i * Kb + (column - qa[i]).  The Krylov dimensions are the run's (replay of
// m_rec); the active-column counts are known on the host, and guard kernels
// check them on the device as in a graph replay (a mismatch raises the
// divergence flag and keeps every index in range).
matex_status recompute_window(matex_ctx* c, int w, int r0, int r1, const std::vector<int>& qa,
                              const std::vector<int>& qb, int g0, int g1,
                              const std::vector<int32_t>& mrec) {
  cudaStream_t st = c->st;
  const int64_t n = c->n;
  const int64_t vstride = (int64_t)kMaxB * n;
  const int Kb = c->tape_Kb;
  const size_t gbytes = sizeof(double) * (size_t)(g1 - g0) * (size_t)n;
  // the block's groups that have not started by the window start from zero
  cudaMemsetAsync(c->Xb + (int64_t)g0 * n, 0, gbytes, st);
  cudaMemsetAsync(c->Zb + (int64_t)g0 * n, 0, gbytes, st);
  cudaMemsetAsync(c->Zpb + (int64_t)g0 * n, 0, gbytes, st);
  {
    const Round& R0 = c->rounds[r0];
    checkpoint_states(c->CK + (c->ck_base[w] + qa[0]) * 2 * n, c->Xb, c->Zb,
                      c->rc_group + R0.begin + qa[0], qb[0] - qa[0], n, true, st);
  }
  for (int r = r0; r < r1; ++r) {
    const int i = r - r0;
    const int K = qb[i] - qa[i];
    if (K <= 0) continue;
    const Round& R = c->rounds[r];
    Round sub = R;
    sub.begin = R.begin + qa[i];
    sub.K = K;
    RoundCols rc = round_cols(c, sub);
    rc.vslot = c->iota_d + (int64_t)i * Kb;
    const int b0 = sub.begin;
    if (r != r0) advance_z(c->Zb, c->Zpb, c->Xb, n, rc, K, n, st);
    build_input_rhs(c->Y, c->ldy, K, rc, c->src, n, st);
    solve_cols(c, c->fG, K);
    scatter_cols(c->Y, c->ldy, K, c->Zpb, n, rc.group, nullptr, n, st);
    scatter_cols(c->Y, c->ldy, K, c->TZp, n, rc.vslot, nullptr, n, st);
    gather_cols(c->Y, c->ldy, K, c->Zpb, n, rc.group, c->c_perm, nullptr, n, st);
    solve_cols(c, c->fG, K);
    scatter_cols(c->Y, c->ldy, K, c->Wb, n, rc.group, nullptr, n, st);
    krylov_start(c->Vb, vstride, c->Xb, c->Zb, c->Wb, n, rc.group, rc.vslot, K, n, c->partials,
                 c->nchunks, st);
    start_finish(c->partials, c->nchunks, K, c->ss, rc.vslot, c->iterA, c->iter_grp, c->d_count,
                 st);
    int32_t* iter = c->iterA;
    int32_t* iter_next = c->iterB;
    auto active = [&](int above) {
      int k = 0;
      for (int q = 0; q < K; ++q) k += mrec[b0 + q] > above ? 1 : 0;
      return k;
    };
    int kit = active(0);
    expect_count(c->d_count, kit, iter, c->iter_grp, rc.vslot, c->d_count + 2, st);
    if (kit > 0) basis_scale(c->Vb, vstride, rc.vslot, iter, kit, 0, c->ss.scale, n, st);
    for (int j = 0; j < c->m_max && kit > 0; ++j) {
      gather_cols(c->Y, c->ldy, kit, c->Vb + (int64_t)j * n, vstride, c->iter_grp, c->c_perm,
                  nullptr, n, st);
      solve_cols(c, c->fM, kit);
      scatter_cols(c->Y, c->ldy, kit, c->Vb + (int64_t)(j + 1) * n, vstride, c->iter_grp, nullptr,
                   n, st);
      scatter_cols(c->Y, c->ldy, kit, c->TA + (int64_t)j * n, (int64_t)kMaxM * n, c->iter_grp,
                   nullptr, n, st);
      for (int pass = 0; pass < 2; ++pass) {
        basis_dots(c->Vb, vstride, rc.vslot, iter, kit, 0, j + 1, j + 1, n, c->partials,
                   c->nchunks, st);
        reduce_dots(c->partials, c->nchunks, kit, j + 1, iter, c->ss, j, pass, st);
        basis_update(c->Vb, vstride, rc.vslot, iter, kit, j + 1, j + 1, c->ss.hbuf, n, st);
      }
      basis_dots(c->Vb, vstride, rc.vslot, iter, kit, j + 1, 1, j + 1, n, c->partials, c->nchunks,
                 st);
      reduce_dots(c->partials, c->nchunks, kit, 1, iter, c->ss, j, 2, st);
      basis_scale(c->Vb, vstride, rc.vslot, iter, kit, j + 1, c->ss.scale, n, st);
      residual_check(c->ss, rc, kit, j, c->gamma, c->tol, c->m_max, c->m_rec, iter, iter_next,
                     c->iter_grp, c->d_count, st);
      std::swap(iter, iter_next);
      kit = active(j + 1);
      expect_count(c->d_count, kit, iter, c->iter_grp, rc.vslot, c->d_count + 2, st);
    }
    tape_small(c->ss, rc, K, c->THt, c->Tbeta, st);
    output_coefficients(c->ss, rc, K, c->gamma, c->dt_out, c->coef, c->n_times, c->yend, st);
    next_state(c->Xb, c->Vb, vstride, c->Zb, c->Zpb, c->Wb, n, rc, c->ss.m, c->yend, K, n, st);
    matex_status s = cuda_check(c, "grad recompute");
    if (s != MATEX_OK) return s;
  }
  return MATEX_OK;
}

// Reverse sweep over the forward's rounds (latest first); per round the
// columns (groups) are handled together, like the forward.  tape = 1 reads
// the run's full tape; tape = 2 goes window by window (latest first) and
// block by block, recomputing each block's segments of the window from the
// window's checkpoint before reversing them.
matex_status run_grad(matex_ctx* c, const double* xbar, double* dc, double* damp) {
  cudaStream_t st = c->st;
  const int64_t n = c->n;
  const int G = c->g_slots;
  const int nrows = c->nrows_out;
  // Krylov dimension per record, from the forward's per-segment record
  std::vector<int32_t> mseg(std::max<int64_t>(1, c->n_segments)), mrec(c->n_records);
  if (cudaMemcpy(mseg.data(), c->m_rec, sizeof(int32_t) * mseg.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return cuda_check(c, "grad m");
  for (int64_t r = 0; r < c->n_records; ++r) mrec[r] = mseg[c->h_segid_all[r]];
  if (!mrec.empty())
    cudaMemcpyAsync(c->mrec_d, mrec.data(), sizeof(int32_t) * mrec.size(), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(c->XBg, 0, sizeof(double) * G * n, st);
  cudaMemsetAsync(c->CARRYg, 0, sizeof(double) * G * n, st);
  cudaMemsetAsync(c->CBg, 0, sizeof(double) * G * n, st);
  cudaMemsetAsync(damp, 0, sizeof(double) * std::max(c->n_src, 1), st);
  SourceTable base = c->src;  // d(B u)/d a_s uses the currents given at setup
  base.pwl_v = c->pwl_base_d;
  matex_status s = MATEX_OK;
  if (c->opts.tape == 1) {
    for (size_t ri = c->rounds.size(); ri-- > 0;) {
      const Round& r = c->rounds[ri];
      s = reverse_round(c, r, 0, r.K, c->rc_vslot + r.begin, mrec, xbar, damp, base);
      if (s != MATEX_OK) return s;
    }
  } else {
    const int W = c->tape_W, Kb = c->tape_Kb;
    const int nr = (int)c->rounds.size();
    const int nwin = (int)c->ck_base.size();
    std::vector<int> qa, qb;
    for (int w = nwin - 1; w >= 0; --w) {
      const int r0 = w * W, r1 = std::min(nr, r0 + W);
      for (int g0 = 0; g0 < G; g0 += Kb) {
        const int g1 = std::min(G, g0 + Kb);
        // the block's columns in each round of the window (columns are in group order)
        qa.assign(r1 - r0, 0);
        qb.assign(r1 - r0, 0);
        bool any = false;
        for (int r = r0; r < r1; ++r) {
          const Round& R = c->rounds[r];
          const int32_t* gb = c->h_group_all.data() + R.begin;
          qa[r - r0] = (int)(std::lower_bound(gb, gb + R.K, g0) - gb);
          qb[r - r0] = (int)(std::lower_bound(gb, gb + R.K, g1) - gb);
          any = any || qb[r - r0] > qa[r - r0];
        }
        if (!any) continue;
        s = recompute_window(c, w, r0, r1, qa, qb, g0, g1, mrec);
        if (s != MATEX_OK) return s;
        for (int r = r1 - 1; r >= r0; --r) {
          const int i = r - r0;
          s = reverse_round(c, c->rounds[r], qa[i], qb[i] - qa[i], c->iota_d + (int64_t)i * Kb,
                            mrec, xbar, damp, base);
          if (s != MATEX_OK) return s;
        }
      }
    }
  }
  // initial states x(0) = G^{-1} B u(0) of the groups whose input is non-zero at t = 0
  const int ng = (int)c->init_groups.size();
  for (int g0 = 0; g0 < ng; g0 += c->ldy) {
    const int K = std::min(c->ldy, ng - g0);
    adj_x0_obs(c->init_groups_d + g0, K, c->XBg, n, xbar, c->out_map, nrows, st);
    gather_cols(c->Y, c->ldy, K, c->XBg, n, c->init_groups_d + g0, nullptr, nullptr, n, st);
    solve_cols(c, c->fG, K);
    adj_init_sources(c->init_groups_d + g0, K, base, c->Y, c->ldy, damp, st);
  }
  adj_csum(c->CBg, G, n, c->perm, dc, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "grad sync");
  s = cuda_check(c, "grad");
  if (s != MATEX_OK) return s;
  int tmp = 0;
  if ((s = read_count(c, &tmp)) != MATEX_OK) return s;
  if (c->opts.tape == 2 && c->h_count[2] != 0)
    return fail(c, MATEX_ERR_STATE,
                "matex_grad: a recomputed segment retired its column at another Krylov step than "
                "the run did");
  return MATEX_OK;
}

}  // namespace

extern "C" {

matex_status matex_grad(matex_ctx* c, const double* xbar, double* dc, double* damp) {
  if (!c) return MATEX_ERR_ARG;
  if (!xbar || !dc || (c->n_src > 0 && !damp)) return fail(c, MATEX_ERR_ARG, "NULL argument");
  if (!c->opts.tape)
    return fail(c, MATEX_ERR_STATE, "matex_grad needs a context set up with tape = 1 or 2");
  if (!c->taped) return fail(c, MATEX_ERR_STATE, "matex_grad needs a preceding batched matex_run");
  cudaMemsetAsync(c->d_count, 0, 4 * sizeof(int32_t), c->st);
  return run_grad(c, xbar, dc, damp);
}

void matex_default_opts(matex_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->col_block = 0;
  o->group_select = -1;
  o->include_dc = 1;
  o->max_width = 1024;
  o->solve_mode = 2;
  o->graph = 1;
}

const char* matex_status_string(matex_status s) {
  switch (s) {
    case MATEX_OK: return "ok";
    case MATEX_ERR_ARG: return "invalid argument";
    case MATEX_ERR_NOT_SPD: return "matrix not symmetric positive definite";
    case MATEX_ERR_CUDA: return "CUDA error";
    case MATEX_ERR_TIMEOUT: return "device wait timed out";
    case MATEX_ERR_NOCONV: return "Krylov iteration did not converge";
    case MATEX_ERR_OOM: return "out of memory";
    case MATEX_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* matex_last_error(const matex_ctx* c) {
  return c ? c->err.c_str() : g_setup_err.c_str();
}

void matex_destroy(matex_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  delete c;
}

matex_status matex_setup(matex_ctx** out, int64_t n, const double* cap, const int64_t* g_rowptr,
                         const int32_t* g_col, const double* g_val, const double* dc_inject,
                         int32_t n_src, const int32_t* src_node, const int32_t* pwl_off,
                         const double* pwl_t, const double* pwl_v, const int32_t* src_group,
                         int32_t n_groups, double gamma, double tol, int32_t m_max, double t_end,
                         double dt_out, const matex_opts* opts, void* stream) {
  g_setup_err.clear();
  auto bad = [&](const std::string& m) {
    g_setup_err = m;
    return MATEX_ERR_ARG;
  };
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (n <= 0 || n > (int64_t)INT32_MAX) return bad("n out of range");
  if (!cap || !g_rowptr || !g_col || !g_val) return bad("C or G pointer is NULL");
  if (n_src < 0 || n_groups < 0) return bad("negative source or group count");
  if (n_src > 0 && (!src_node || !pwl_off || !pwl_t || !pwl_v || !src_group))
    return bad("source arrays are NULL");
  if (!(gamma > 0) || !(tol > 0) || m_max < 1 || m_max > kMaxM || !(t_end > 0) || !(dt_out > 0))
    return bad("gamma/tol/m_max/t_end/dt_out out of range");
  for (int64_t i = 0; i < n; ++i)
    if (!(cap[i] > 0) || !std::isfinite(cap[i])) return bad("capacitance must be positive");
  if (g_rowptr[0] != 0) return bad("G row pointer must start at 0");
  for (int64_t i = 0; i < n; ++i) {
    if (g_rowptr[i + 1] < g_rowptr[i]) return bad("G row pointers decrease");
    bool diag = false;
    for (int64_t p = g_rowptr[i]; p < g_rowptr[i + 1]; ++p) {
      if (g_col[p] < 0 || g_col[p] >= n) return bad("G column index out of range");
      if (!std::isfinite(g_val[p])) return bad("G has a non-finite value");
      if (p > g_rowptr[i] && g_col[p] <= g_col[p - 1]) return bad("G columns must be sorted and unique");
      if (g_col[p] == i) diag = true;
    }
    if (!diag) return bad("G row without a diagonal entry");
  }
  // symmetry
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = g_rowptr[i]; p < g_rowptr[i + 1]; ++p) {
      const int32_t j = g_col[p];
      const int32_t* b = g_col + g_rowptr[j];
      const int32_t* e = g_col + g_rowptr[j + 1];
      const int32_t* f = std::lower_bound(b, e, (int32_t)i);
      if (f == e || *f != i || g_val[g_rowptr[j] + (f - b)] != g_val[p]) return bad("G is not symmetric");
    }
  for (int32_t s = 0; s < n_src; ++s) {
    if (src_node[s] < 0 || src_node[s] >= n) return bad("source node out of range");
    if (src_group[s] < 0 || src_group[s] >= n_groups) return bad("source group out of range");
    if (pwl_off[s + 1] <= pwl_off[s]) return bad("source without breakpoints");
    for (int32_t p = pwl_off[s]; p < pwl_off[s + 1]; ++p) {
      if (!std::isfinite(pwl_t[p]) || !std::isfinite(pwl_v[p])) return bad("non-finite PWL data");
      if (p > pwl_off[s] && !(pwl_t[p] > pwl_t[p - 1])) return bad("PWL times must increase");
    }
  }
  if (pwl_off && pwl_off[0] != 0) return bad("pwl_off must start at 0");
  matex_opts o;
  matex_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_width <= 0) o.max_width = 1024;
  if (o.tape < 0 || o.tape > 2) return bad("tape must be 0, 1 or 2");
  if (o.tape_window < 0 || o.tape_block < 0) return bad("tape_window and tape_block must be >= 0");
  if (o.tape && o.group_select >= 0) return bad("tape needs all groups (group_select = -1)");
  if (o.solve_mode < 0 || o.solve_mode > 2) return bad("solve_mode must be 0, 1 or 2");
  if (o.krylov < 0 || o.krylov > 2) return bad("krylov must be 0, 1 or 2");
  if (o.tape && o.krylov != 0) return bad("the adjoint tape follows the rational Krylov space only");
  if (!std::isfinite(o.tail_eps) || o.tail_eps < 0.0) return bad("tail_eps must be finite and >= 0");
  if (o.tape && o.tail_eps > 0.0) return bad("the adjoint tape follows exact runs only (tail_eps 0)");
  if (o.recombine < 0 || o.recombine > 1) return bad("recombine must be 0 or 1");
  if (o.decompose < 0 || o.decompose > 1) return bad("decompose must be 0 or 1");
  if (o.decompose == 1 && (o.tape || o.group_select >= 0))
    return bad("decompose = 1 (ramps) needs tape = 0 and group_select = -1");
  if (o.col_block != 0 && o.col_block != 1 && o.col_block != 2 && o.col_block != 4 && o.col_block != 8)
    return bad("col_block must be 0, 1, 2, 4 or 8");
  if (o.resident < 0 || o.resident > 3) return bad("resident must be 0, 1, 2 or 3");
  if (o.tc_solve < 0 || o.tc_solve > 2) return bad("tc_solve must be 0, 1 or 2");
  if (o.tc_min_width != 0 && o.tc_min_width < 32) return bad("tc_min_width must be 0 or >= 32");
  if (o.single_column < 0 || o.single_column > 2) return bad("single_column must be 0, 1 or 2");
  if (o.resident >= 2 && (o.krylov == 2 || o.tape || o.tail_eps > 0.0 || n > kResidentMaxN))
    return bad("resident rounds need n <= 8192, krylov 0 or 1, tape 0 and tail_eps 0");
  if (o.group_select >= n_groups) return bad("group_select out of range");
  if (o.n_rows < 0 || (o.n_rows > 0 && !o.rows)) return bad("row list missing");
  for (int32_t r = 0; r < o.n_rows; ++r)
    if (o.rows[r] < 0 || o.rows[r] >= n) return bad("output row out of range");

  matex_ctx* c = new (std::nothrow) matex_ctx();
  if (!c) return MATEX_ERR_OOM;
  c->opts = o;
  c->st = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  c->n = n;
  c->n_src = n_src;
  c->n_groups = n_groups;
  c->gamma = gamma;
  c->tol = tol;
  c->m_max = m_max;
  c->dt_out = dt_out;
  const int N = (int)std::llround(t_end / dt_out);
  if (N < 1) { delete c; return bad("t_end / dt_out must be >= 1"); }
  c->n_times = N + 1;
  c->T = (double)N * dt_out;
  RampProblem ramps;
  if (o.decompose == 1 && n_src > 0) {
    // from here on the problem is the ramp-decomposed one
    ramp_transform(n_src, src_node, pwl_off, pwl_t, pwl_v, src_group, c->T, ramps);
    n_src = (int32_t)ramps.node.size();
    src_node = ramps.node.data();
    pwl_off = ramps.off.data();
    pwl_t = ramps.t.data();
    pwl_v = ramps.v.data();
    src_group = ramps.grp.data();
    n_groups = ramps.ngroups;
    c->n_src = n_src;
    c->n_groups = n_groups;
  }
  if (o.n_rows > 0) c->rows.assign(o.rows, o.rows + o.n_rows);
  c->nrows_out = o.n_rows > 0 ? o.n_rows : (int32_t)n;
  c->opts.rows = nullptr;
  c->opts.replay_m = nullptr;

  // ---- ordering, symbolic, numeric ------------------------------------
  double t = now_ms();
  c->c_host.assign(cap, cap + n);
  c->g_rowptr_h.assign(g_rowptr, g_rowptr + n + 1);
  c->g_col_h.assign(g_col, g_col + g_rowptr[n]);
  c->g_val_h.assign(g_val, g_val + g_rowptr[n]);
  CsrSym A{n, g_rowptr, g_col, g_val};
  std::vector<int32_t> nd;
  std::string e = nested_dissection(A, nd);
  if (e.empty()) e = symbolic_analysis(A, nd, o.max_width, c->S);
  if (!e.empty()) { c->err = e; g_setup_err = e; delete c; return MATEX_ERR_ARG; }
  c->setup_stats.setup_order_ms = now_ms() - t;
  t = now_ms();
  Numeric NM, NG;
  {
    // the two factorisations are independent: run them side by side
    std::string eg;
    std::thread tg([&] { eg = numeric_ldlt(A, nullptr, 1.0, c->S, NG); });
    e = numeric_ldlt(A, cap, gamma, c->S, NM);
    tg.join();
    if (e.empty()) e = eg;
  }
  if (!e.empty()) { g_setup_err = e; delete c; return MATEX_ERR_NOT_SPD; }
  c->setup_stats.setup_factor_ms = now_ms() - t;
  c->setup_stats.nnz_L = c->S.nnz_L;
  c->setup_stats.nnz_L_exact = c->S.nnz_L_exact;
  c->setup_stats.n_supernodes = c->S.nsup;
  c->setup_stats.n_levels = (int32_t)c->S.level_ptr.size() - 1;

  // ---- groups, segments, rounds ------------------------------------------
  for (int32_t g = 0; g < n_groups; ++g)
    if (o.group_select < 0 || o.group_select == g) c->sel_groups.push_back(g);
  std::vector<std::vector<int32_t>> gsrc(n_groups);
  for (int32_t s = 0; s < n_src; ++s) gsrc[src_group[s]].push_back(s);
  // A segment whose group has injected nothing since t = 0 and injects nothing
  // on it has x = z = z' = w = 0 and contributes exactly zero: it is recorded
  // (m = 0) but never solved.  A group whose input is zero at t = 0 starts
  // from x = 0 without a solve.
  struct Seg { int32_t g, j, obeg, nout; double l0, len, hfirst, lprev; int64_t id; bool zero; };
  std::vector<std::vector<Seg>> per_group;
  int64_t segid = 0;
  size_t max_segs = 0;
  std::vector<int32_t> init_groups;
  for (int32_t g : c->sel_groups) {
    std::vector<double> lts = group_lts(gsrc[g], pwl_off, pwl_t, c->T);
    std::vector<Seg> segs;
    bool quiet = group_input_zero(gsrc[g], pwl_off, pwl_t, pwl_v, 0.0);
    if (!quiet) init_groups.push_back(g);
    c->ginit_h.push_back(quiet ? 0 : 1);
    c->glts_h.push_back(lts);
    for (size_t j = 0; j + 1 < lts.size(); ++j) {
      Seg sg;
      sg.g = g;
      sg.j = (int32_t)j;
      sg.l0 = lts[j];
      sg.len = lts[j + 1] - lts[j];
      sg.lprev = j > 0 ? lts[j] - lts[j - 1] : 0.0;
      quiet = quiet && group_input_zero(gsrc[g], pwl_off, pwl_t, pwl_v, lts[j]) &&
              group_input_zero(gsrc[g], pwl_off, pwl_t, pwl_v, lts[j + 1]);
      sg.zero = quiet;
      // outputs with l_j < t_o <= l_{j+1}
      int ob = -1, cnt = 0;
      int o0 = std::max(0, (int)std::floor(lts[j] / dt_out) - 1);
      for (int oo = o0; oo < c->n_times; ++oo) {
        const double to = (double)oo * dt_out;
        if (to > lts[j + 1]) break;
        if (to > lts[j]) {
          if (ob < 0) ob = oo;
          cnt++;
        }
      }
      sg.obeg = ob < 0 ? 0 : ob;
      sg.nout = cnt;
      sg.hfirst = cnt > 0 ? (double)sg.obeg * dt_out - lts[j] : sg.len;
      sg.id = segid++;
      segs.push_back(sg);
    }
    max_segs = std::max(max_segs, segs.size());
    std::vector<char> zf;
    for (const Seg& sg : segs) zf.push_back(sg.zero ? 1 : 0);
    c->gzero_h.push_back(std::move(zf));
    per_group.push_back(std::move(segs));
  }
  c->n_segments = segid;
  c->gsrc_h = gsrc;
  c->pwl_off_h.assign(pwl_off, pwl_off + n_src + 1);
  c->pwl_t_h.assign(pwl_t, pwl_t + pwl_off[n_src]);
  std::vector<int32_t> h_group, h_sgroup, h_seg, h_obeg, h_nout;
  std::vector<double> h_l0, h_len, h_hfirst, h_lprev;
  std::vector<int64_t> h_segid;
  int Kmax = 1;
  const int nsel = (int)per_group.size();
  int bsize = std::max(nsel, 1);
  if (o.decompose == 1 && nsel > kRampBatch) {
    // ramp columns in batches whose state and basis slots fit in memory
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double per_slot = 8.0 * (kMaxB + 4.0) * (double)n;
    bsize = (int)std::min<double>(kRampBatch, std::max(8.0, 0.35 * (double)free_b / per_slot));
    bsize = std::max(8, bsize & ~7);
  }
  std::vector<int32_t> init_slots;
  std::vector<int32_t> init_src;
  for (int b0 = 0; b0 < nsel; b0 += bsize) {
    const int b1 = std::min(nsel, b0 + bsize);
    matex_ctx::Batch bt;
    bt.r0 = (int32_t)c->rounds.size();
    bt.i0 = (int32_t)init_src.size();
    for (int k = b0; k < b1; ++k)
      if (c->ginit_h[k]) {
        init_src.push_back(c->sel_groups[k]);
        init_slots.push_back(bsize < nsel ? k - b0 : c->sel_groups[k]);
      }
    bt.ni = (int32_t)init_src.size() - bt.i0;
    size_t bmax = 0;
    for (int k = b0; k < b1; ++k) bmax = std::max(bmax, per_group[k].size());
  for (size_t r = 0; r < bmax; ++r) {
    Round rd;
    rd.begin = (int32_t)h_group.size();
    rd.obeg_min = c->n_times;
    rd.oend_max = 0;
    for (int k = b0; k < b1; ++k) {
      const std::vector<Seg>& segs = per_group[k];
      if (r >= segs.size() || segs[r].zero) continue;
      const Seg& sg = segs[r];
      h_group.push_back(bsize < nsel ? k - b0 : sg.g);
      h_sgroup.push_back(sg.g);
      h_seg.push_back(sg.j);
      h_obeg.push_back(sg.obeg);
      h_nout.push_back(sg.nout);
      h_l0.push_back(sg.l0);
      h_len.push_back(sg.len);
      h_hfirst.push_back(sg.hfirst);
      h_lprev.push_back(sg.lprev);
      h_segid.push_back(sg.id);
      if (sg.nout > 0) {
        rd.obeg_min = std::min(rd.obeg_min, sg.obeg);
        rd.oend_max = std::max(rd.oend_max, sg.obeg + sg.nout);
      }
    }
    rd.K = (int32_t)h_group.size() - rd.begin;
    Kmax = std::max(Kmax, rd.K);
    if (rd.K > 0) c->rounds.push_back(rd);
  }
    bt.r1 = (int32_t)c->rounds.size();
    c->batches.push_back(bt);
  }
  c->g_slots = bsize < nsel ? bsize : std::max(n_groups, 1);
  init_groups = init_src;
  c->init_groups = init_groups;
  c->Kmax = Kmax;
  c->h_nout_all = h_nout;
  c->h_segid_all = h_segid;
  c->h_group_all = h_group;
  std::vector<int32_t> ev_o_h, ev_q_h;
  for (Round& rd : c->rounds) {
    std::vector<char> cov(c->n_times, 0);
    int cnt = 0;
    double held = 0.0;
    std::vector<std::pair<int32_t, int32_t>> ev;
    for (int q = 0; q < rd.K; ++q) {
      const int ob = h_obeg[rd.begin + q], no = h_nout[rd.begin + q];
      held += no;
      if (no > 0) {
        ev.push_back({ob, q + 1});
        ev.push_back({ob + no, -(q + 1)});
      }
      for (int o = ob; o < ob + no; ++o)
        if (!cov[o]) { cov[o] = 1; cnt++; }
    }
    c->round_cover.push_back(cnt);
    const int span = rd.oend_max - rd.obeg_min;
    rd.cover = span > 0 ? held / ((double)rd.K * span) : 0.0;
    std::stable_sort(ev.begin(), ev.end(),
                     [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                       return a.first < b.first;
                     });
    rd.ev_begin = (int32_t)ev_o_h.size();
    rd.nev = (int32_t)ev.size();
    for (const auto& x : ev) {
      ev_o_h.push_back(x.first);
      ev_q_h.push_back(x.second);
    }
  }
  c->offd_rows = c->S.sup_rowptr[c->S.nsup] - c->S.n;
  // the same column records, one group at a time in time order
  {
    std::vector<std::vector<int32_t>> by_group(n_groups);
    for (const Round& rd : c->rounds)
      for (int q = 0; q < rd.K; ++q) by_group[h_sgroup[rd.begin + q]].push_back(rd.begin + q);
    for (int32_t g = 0; g < n_groups; ++g)
      for (int32_t rec : by_group[g]) {
        Round one;
        one.begin = rec;
        one.K = 1;
        one.obeg_min = h_nout[rec] > 0 ? h_obeg[rec] : c->n_times;
        one.oend_max = h_nout[rec] > 0 ? h_obeg[rec] + h_nout[rec] : 0;
        c->serial_rounds.push_back(one);
        c->serial_cover.push_back(h_nout[rec]);
      }
  }
  if (opts && opts->replay_m) {
    if (opts->n_replay != c->n_segments) {
      g_setup_err = "replay_m length differs from the number of segments";
      delete c;
      return MATEX_ERR_ARG;
    }
    c->replay.assign(opts->replay_m, opts->replay_m + opts->n_replay);
  }

  // ---- upload --------------------------------------------------------------
  t = now_ms();
  bool ok = true;
  const Symbolic& S = c->S;
  int32_t *sup_first, *sup_rows, *sup_parent;
  int64_t *sup_rowptr, *pan_off;
  ok = ok && c->upload(sup_first, S.sup_first.data(), S.sup_first.size());
  ok = ok && c->upload(sup_parent, S.sup_parent.data(), S.sup_parent.size());
  ok = ok && c->upload(sup_rowptr, S.sup_rowptr.data(), S.sup_rowptr.size());
  ok = ok && c->upload(sup_rows, S.sup_rows.data(), S.sup_rows.size());
  ok = ok && c->upload(pan_off, S.pan_off.data(), S.pan_off.size());
  auto up_factor = [&](const Numeric& Nm, DevFactor& F) {
    double *dinv, *pcm, *prm;
    bool k = c->upload(dinv, Nm.dinv.data(), Nm.dinv.size()) &&
             c->upload(pcm, Nm.pan_cm.data(), Nm.pan_cm.size()) &&
             c->upload(prm, Nm.pan_rm.data(), Nm.pan_rm.size());
    F = DevFactor{sup_first, sup_parent, sup_rowptr, sup_rows, pan_off, dinv, pcm, prm,
                  nullptr, nullptr, nullptr, nullptr};
    return k;
  };
  ok = ok && up_factor(NM, c->fM) && up_factor(NG, c->fG);
  {
    std::vector<double> cp(n), dp(n, 0.0);
    for (int64_t k = 0; k < n; ++k) {
      cp[k] = cap[S.perm[k]];
      if (dc_inject) dp[k] = dc_inject[S.perm[k]];
    }
    ok = ok && c->upload(c->c_perm, cp.data(), n);
    if (dc_inject) ok = ok && c->upload(c->dc_perm, dp.data(), n);
    ok = ok && c->upload(c->perm, S.perm.data(), n);
    std::vector<int32_t> omap(c->nrows_out);
    for (int32_t r = 0; r < c->nrows_out; ++r)
      omap[r] = c->rows.empty() ? S.iperm[r] : S.iperm[c->rows[r]];
    ok = ok && c->upload(c->out_map, omap.data(), omap.size());
  }
  {
    std::vector<int32_t> gptr(n_groups + 1, 0), gs;
    for (int32_t g = 0; g < n_groups; ++g) {
      gptr[g + 1] = gptr[g] + (int32_t)gsrc[g].size();
      gs.insert(gs.end(), gsrc[g].begin(), gsrc[g].end());
    }
    std::vector<int32_t> node(n_src);
    for (int32_t s = 0; s < n_src; ++s) node[s] = S.iperm[src_node[s]];
    const size_t npwl = n_src ? (size_t)pwl_off[n_src] : 0;
    int32_t *gp, *gsd, *nd_d, *po;
    double* pt;
    ok = ok && c->upload(gp, gptr.data(), gptr.size()) && c->upload(gsd, gs.data(), gs.size()) &&
         c->upload(nd_d, node.data(), node.size());
    std::vector<int32_t> poff(pwl_off ? pwl_off : nullptr, pwl_off ? pwl_off + n_src + 1 : nullptr);
    if (poff.empty()) poff.push_back(0);
    ok = ok && c->upload(po, poff.data(), poff.size()) && c->upload(pt, pwl_t, npwl) &&
         c->upload(c->pwl_v_d, pwl_v, npwl) && c->upload(c->pwl_base_d, pwl_v, npwl);
    c->pwl_v_host_shape.resize(npwl);
    c->src = SourceTable{gp, gsd, nd_d, po, pt, c->pwl_v_d};
  }
  ok = ok && c->upload(c->sel_groups_d, c->sel_groups.data(), c->sel_groups.size());
  ok = ok && c->upload(c->init_groups_d, c->init_groups.data(), c->init_groups.size());
  ok = ok && c->upload(c->init_slots_d, init_slots.data(), init_slots.size());
  ok = ok && c->upload(c->rc_sgroup, h_sgroup.data(), h_sgroup.size());
  ok = ok && c->upload(c->ev_o_d, ev_o_h.data(), ev_o_h.size()) &&
       c->upload(c->ev_q_d, ev_q_h.data(), ev_q_h.size());
  std::vector<int32_t> h_vslot(h_group.size());
  for (size_t r = 0; r < h_group.size(); ++r) h_vslot[r] = o.tape == 1 ? (int32_t)r : h_group[r];
  ok = ok && c->upload(c->rc_vslot, h_vslot.data(), h_vslot.size());
  ok = ok && c->upload(c->rc_group, h_group.data(), h_group.size()) &&
       c->upload(c->rc_seg, h_seg.data(), h_seg.size()) &&
       c->upload(c->rc_obeg, h_obeg.data(), h_obeg.size()) &&
       c->upload(c->rc_nout, h_nout.data(), h_nout.size()) &&
       c->upload(c->rc_l0, h_l0.data(), h_l0.size()) &&
       c->upload(c->rc_len, h_len.data(), h_len.size()) &&
       c->upload(c->rc_hfirst, h_hfirst.data(), h_hfirst.size()) &&
       c->upload(c->rc_lprev, h_lprev.data(), h_lprev.size()) &&
       c->upload(c->rc_segid, h_segid.data(), h_segid.size());
  if (!c->replay.empty()) ok = ok && c->upload(c->replay_d, c->replay.data(), c->replay.size());
  // work buffers
  c->ldy = roundup8(std::max({Kmax, 8, std::min<int>(n_groups, 256)}));
  c->ts_minw = o.tc_solve == 1 ? 0 : (o.tc_min_width > 0 ? o.tc_min_width : kTsMinWidth);
  ok = ok && plan_levels(c);
  c->nchunks = (int)((n + kChunk - 1) / kChunk);
  const size_t G = (size_t)c->g_slots;
  c->n_records = (int64_t)h_group.size();
  if (ok && o.decompose == 1) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double need = 8.0 * (double)G * (kMaxB + 4.0) * (double)n;
    if (need > 0.9 * (double)free_b) {
      char msg[256];
      std::snprintf(msg, sizeof(msg),
                    "decompose = 1: %d ramps need %.1f GB of Krylov bases and states, %.1f GB free",
                    (int)G, need / 1e9, (double)free_b / 1e9);
      g_setup_err = msg;
      delete c;
      return MATEX_ERR_OOM;
    }
  }
  if (ok && o.tape == 2) {
    // what the run itself holds, then the plan within most of the rest
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double nd = (double)n;
    const double run_b = 8.0 * (2.0 * nd * c->ldy + (double)G * kMaxB * nd + 4.0 * G * nd +
                                (double)c->n_times * nd + (double)Kmax * c->n_times * kCoefLd +
                                (double)Kmax * kMaxB * c->nchunks);
    const double budget = 0.85 * ((double)free_b - run_b);
    const TapePlan tp = plan_tape(c->rounds, n, (int)G, Kmax, c->n_times, c->nrows_out, budget,
                                  o.tape_window, o.tape_block);
    if (!tp.W) {
      g_setup_err = "tape = 2: no checkpoint window and block fit the free device memory";
      delete c;
      return MATEX_ERR_OOM;
    }
    c->tape_W = tp.W;
    c->tape_Kb = tp.Kb;
    int64_t slot = 0;
    for (size_t r = 0; r < c->rounds.size(); r += (size_t)tp.W) {
      c->ck_base.push_back(slot);
      slot += c->rounds[r].K;
    }
    ok = c->alloc(c->CK, (size_t)std::max<int64_t>(1, slot) * 2 * n);
    c->tape_bytes = (int64_t)tp.bytes;
  }
  const size_t vslots = o.tape == 1 ? (size_t)std::max<int64_t>(1, c->n_records)
                        : o.tape == 2 ? std::max(G, (size_t)c->tape_W * c->tape_Kb)
                                      : G;
  ok = ok && c->alloc(c->Y, (size_t)n * c->ldy) && c->alloc(c->Y2, (size_t)n * c->ldy) && c->alloc(c->Vb, vslots * kMaxB * n) &&
       c->alloc(c->Zb, G * n) && c->alloc(c->Zpb, G * n) && c->alloc(c->Wb, G * n) &&
       c->alloc(c->Xb, G * n) && c->alloc(c->Xp, (size_t)c->n_times * n) && c->alloc(c->xdc, n) &&
       c->alloc(c->partials, (size_t)Kmax * kMaxB * c->nchunks) &&
       c->alloc(c->ss.Ht, (size_t)Kmax * kMaxB * kMaxM) && c->alloc(c->ss.beta, Kmax) &&
       c->alloc(c->ss.m, Kmax) && c->alloc(c->ss.status, Kmax) &&
       c->alloc(c->ss.hbuf, (size_t)Kmax * kMaxB) && c->alloc(c->ss.scale, Kmax) &&
       c->alloc(c->iterA, Kmax) && c->alloc(c->iterB, Kmax) && c->alloc(c->iter_grp, Kmax) &&
       c->alloc(c->d_count, 4) && c->alloc(c->coef, (size_t)Kmax * c->n_times * kCoefLd) &&
       c->alloc(c->yend, (size_t)Kmax * kMaxM) &&
       c->alloc(c->tcut, (size_t)Kmax * 2) && c->alloc(c->pbound, (size_t)Kmax * 2) && c->alloc(c->m_rec, std::max<int64_t>(1, c->n_segments)) &&
       c->alloc(c->st_rec, std::max<int64_t>(1, c->n_segments));
  if (ok && cudaMallocHost(&c->h_count, 4 * sizeof(int32_t)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(c->d_count, 0, 4 * sizeof(int32_t)) != cudaSuccess) ok = false;
  if (ok) c->fM.abort = c->fG.abort = c->d_count + 2;
  if (ok && o.tape) {
    // tape 1: one entry per record, reverse launches as wide as a round;
    // tape 2: one entry per window-tape slot, launches as wide as a block
    const size_t R = o.tape == 1 ? (size_t)std::max<int64_t>(1, c->n_records)
                                 : (size_t)c->tape_W * c->tape_Kb;
    const size_t KM = o.tape == 1 ? (size_t)Kmax : (size_t)c->tape_Kb;
    if (o.tape == 1)
      c->tape_bytes = (int64_t)(8.0 * (double)R * ((kMaxM + 1) * (double)n + kMaxB * (double)n));
    std::vector<int32_t> iota(std::max<size_t>(std::max(Kmax, 1), R));
    for (int q = 0; q < (int)iota.size(); ++q) iota[q] = q;
    ok = c->alloc(c->TA, R * kMaxM * n) && c->alloc(c->TZp, R * n) &&
         c->alloc(c->THt, R * kMaxB * kMaxM) && c->alloc(c->Tbeta, R) &&
         c->alloc(c->AW, KM * kWSlots * n) && c->alloc(c->XBg, G * n) && c->alloc(c->CARRYg, G * n) &&
         c->alloc(c->CBg, G * n) && c->alloc(c->YBO, KM * c->n_times * kCoefLd) &&
         c->alloc(c->YOUT, KM * c->n_times * kCoefLd) && c->alloc(c->YBL, KM * kMaxB) &&
         c->alloc(c->YL, KM * kMaxM) && c->alloc(c->HTB, KM * kMaxB * kMaxM) &&
         c->alloc(c->BETAB, KM) && c->alloc(c->D1, KM * kMaxB) && c->alloc(c->HD, KM * kMaxB) &&
         c->alloc(c->D0, KM * kMaxB) && c->alloc(c->S1, KM * c->nrows_out) &&
         c->alloc(c->S2, KM * c->nrows_out) && c->upload(c->iota_d, iota.data(), iota.size()) &&
         c->alloc(c->mrec_d, std::max<int64_t>(1, c->n_records)) &&
         c->alloc(c->act_d, KM * (kMaxM + 1));
    adj_set_limits();
  }
  if (!ok) {
    cudaGetLastError();
    g_setup_err = "device allocation or upload failed";
    delete c;
    return MATEX_ERR_OOM;
  }
  set_small_smem_limits();
  if (o.recombine == 0 && o.tail_eps == 0.0) {
    // tensor-core recombination scratch, sized once for rounds of up to
    // kdim_cap basis vectors (never regrown: recorded graphs keep pointers)
    int cap = std::min(Kmax * m_max, kTcMaxKdim);
    cap = (cap + 31) & ~31;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    while (cap > 32 && (double)tc_slices_bytes(n, cap, c->n_times) > 0.3 * (double)free_b) cap -= 32;
    if (cap >= kTcMinKdim &&
        (double)tc_slices_bytes(n, cap, c->n_times) <= 0.3 * (double)free_b) {
      unsigned char* sl = nullptr;
      int64_t* km = nullptr;
      int32_t* kq = nullptr;
      double *rsc = nullptr, *csc = nullptr;
      const size_t ncol = ((size_t)c->n_times + 47) / 48 * 48;
      if (c->alloc(sl, tc_slices_bytes(n, cap, c->n_times)) && c->alloc(km, cap) &&
          c->alloc(kq, cap) && c->alloc(rsc, n) && c->alloc(csc, ncol)) {
        c->tc = TcScratch{sl, km, kq, rsc, csc, c->d_count + 1, cap};
        tc_set_limits();
      } else {
        cudaGetLastError();  // no room: the FP64 recombination serves every round
      }
    }
  }
  c->ss.krylov = o.krylov;
  c->ss.rscale = o.krylov == 1 ? 1.0 / gamma : o.krylov == 2 ? gamma : 1.0;
  if (o.krylov == 2 && !ensure_g_csr(c)) {
    g_setup_err = "device allocation or upload failed";
    delete c;
    return MATEX_ERR_OOM;
  }
  if (o.solve_mode == 2 && o.col_block == 0) autotune_levels(c);
  if (o.solve_mode == 2) autotune_solve(c);
  if (c->ts_minw > 0 && o.solve_mode != 0) {
    if (plan_ts(c)) autotune_ts(c);
    cudaGetLastError();
  }
  c->setup_stats.tc_solve_supernodes = c->ts_n;
  c->setup_stats.tc_solve_min_cols = c->ts_min_cols;
  if (o.single_column == 2 || (o.single_column == 0 && o.solve_mode == 2)) {
    autotune_k1(c);
    cudaGetLastError();
  }
  c->setup_stats.single_column = c->k1_use ? 1 : 0;
  if (o.resident != 1 && o.krylov != 2 && o.tape == 0 && o.tail_eps == 0.0 &&
      n <= kResidentMaxN) {
    // resident rounds: one CTA's solve pair against the batched path's
    // single-column pair (in its tuned launch mode), best of five each
    if (plan_resident(c, kResidentThreads) && resident_fits(n, c->rplan) &&
        resident_set_limits(n, c->rplan)) {
      c->resident_ok = true;
      cudaMemsetAsync(c->Y, 0, sizeof(double) * (size_t)n * c->ldy, c->st);
      const ResFactor& R1 = o.krylov == 1 ? c->rG : c->rM;
      const DevFactor& F1 = o.krylov == 1 ? c->fG : c->fM;
      c->res_pair_ms = resident_time_solve(R1, c->rplan, c->Y, c->Y2, n, c->st, 5);
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      solve_cols(c, F1, 1);
      float best = 1e30f;
      for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, c->st);
        solve_cols(c, F1, 1);
        cudaEventRecord(e1, c->st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c->lvl_pair_ms = best;
      c->resident = c->res_pair_ms > 0.f && (o.resident >= 2 || c->res_pair_ms <= 2.f * best);
      // room for every record's z' and w (at most a quarter of the free
      // memory): the input solves then run ahead of the rounds (not with
      // resident = 3, which keeps them in the round kernels)
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      const double need = 16.0 * (double)c->n_records * (double)n;
      if (c->resident && o.resident != 3 && c->n_records > 0 && need <= 0.25 * (double)free_b &&
          !(c->alloc(c->pre_zp, (size_t)c->n_records * n) &&
            c->alloc(c->pre_w, (size_t)c->n_records * n)))
        c->pre_zp = c->pre_w = nullptr;
    }
    cudaGetLastError();
  }
  if (o.resident >= 2 && !c->resident) {
    g_setup_err = "resident rounds do not fit this device (shared memory or launch failed)";
    delete c;
    return MATEX_ERR_ARG;
  }
  c->setup_stats.resident = c->resident ? 1 : 0;
  {
    // Load, here, everything matex_solve_noalloc touches on this device: the
    // module that holds its static scratch array (under lazy module loading
    // the array is allocated when its module is first loaded) and every solve
    // kernel.  Its first call then allocates nothing.  A failure here is left
    // for that call to report.
    void* scratch = nullptr;
    std::string serr;
    if (noalloc_scratch(c->device, &scratch, serr) != MATEX_OK) cudaGetLastError();
    preload_solve_kernels();
  }
  cudaMemset(c->Vb, 0, sizeof(double) * vslots * kMaxB * n);
  cudaMemset(c->Xb, 0, sizeof(double) * G * n);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    g_setup_err = std::string("setup: ") + cudaGetErrorString(cudaGetLastError());
    delete c;
    return MATEX_ERR_CUDA;
  }
  c->setup_stats.setup_upload_ms = now_ms() - t;
  c->setup_stats.tape_window = c->tape_W;
  c->setup_stats.tape_block = c->tape_Kb;
  c->setup_stats.tape_bytes = c->tape_bytes;
  *out = c;
  return MATEX_OK;
}

matex_status matex_run(matex_ctx* c, double* x_out, matex_stats* stats) {
  if (!c) return MATEX_ERR_ARG;
  if (!x_out) return fail(c, MATEX_ERR_ARG, "x_out is NULL");
  return run_device(c, x_out, stats);
}

matex_status matex_set_caps(matex_ctx* c, const double* cap) {
  if (!c) return MATEX_ERR_ARG;
  if (!cap) return fail(c, MATEX_ERR_ARG, "capacitances are NULL");
  for (int64_t i = 0; i < c->n; ++i)
    if (!(cap[i] > 0) || !std::isfinite(cap[i])) return fail(c, MATEX_ERR_ARG, "capacitance must be positive");
  const double t = now_ms();
  CsrSym A{c->n, c->g_rowptr_h.data(), c->g_col_h.data(), c->g_val_h.data()};
  Numeric NM;
  std::string e = numeric_ldlt(A, cap, c->gamma, c->S, NM);
  if (!e.empty()) return fail(c, MATEX_ERR_NOT_SPD, e);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "set_caps sync");
  std::vector<double> cp(c->n);
  for (int64_t k = 0; k < c->n; ++k) cp[k] = cap[c->S.perm[k]];
  bool ok = cudaMemcpy(const_cast<double*>(c->fM.dinv), NM.dinv.data(), sizeof(double) * NM.dinv.size(),
                       cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(const_cast<double*>(c->fM.pan_cm), NM.pan_cm.data(),
                       sizeof(double) * NM.pan_cm.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(const_cast<double*>(c->fM.pan_rm), NM.pan_rm.data(),
                       sizeof(double) * NM.pan_rm.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->c_perm, cp.data(), sizeof(double) * c->n, cudaMemcpyHostToDevice) ==
                cudaSuccess;
  if (!ok) return cuda_check(c, "set_caps upload");
  if (c->ts_n > 0) {
    // the tensor-core slices of the refactored C + gamma G
    ts_split_panels(c->fM, c->ts_sups, c->ts_n, c->ts_mtf, true, c->tsA[0][0], c->tsR[0][0], c->st);
    ts_split_panels(c->fM, c->ts_sups, c->ts_n, c->ts_mtb, false, c->tsA[0][1], c->tsR[0][1], c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "set_caps slices");
  }
  if (c->resident_ok) {
    // the resident copy of the refactored C + gamma G
    resident_store(c->fM, c->rsup, c->S.nsup, const_cast<double*>(c->rM.fpan),
                   const_cast<double*>(c->rM.bpan), c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "set_caps resident copy");
  }
  c->c_host.assign(cap, cap + c->n);
  c->taped = false;
  c->tr_h = 0.0;  // the trapezoidal factor C + h/2 G is refactored on its next use
  c->setup_stats.setup_factor_ms = now_ms() - t;
  return MATEX_OK;
}

// True when the currents pwl_v keep zero every segment that setup skipped as
// identically zero, and keep zero at t = 0 every group that starts from x = 0.
static bool zero_pattern_kept(const matex_ctx* c, const double* pwl_v) {
  const int32_t* off = c->pwl_off_h.data();
  const double* pt = c->pwl_t_h.data();
  for (size_t k = 0; k < c->sel_groups.size(); ++k) {
    const std::vector<int32_t>& srcs = c->gsrc_h[c->sel_groups[k]];
    const std::vector<double>& lts = c->glts_h[k];
    bool quiet = group_input_zero(srcs, off, pt, pwl_v, 0.0);
    if (!quiet && !c->ginit_h[k]) return false;
    for (size_t j = 0; j + 1 < lts.size() && quiet; ++j) {
      quiet = group_input_zero(srcs, off, pt, pwl_v, lts[j]) &&
              group_input_zero(srcs, off, pt, pwl_v, lts[j + 1]);
      if (!quiet && c->gzero_h[k][j]) return false;
    }
  }
  return true;
}

static matex_status check_sources(matex_ctx* c, const double* pwl_v_host) {
  for (size_t i = 0; i < c->pwl_v_host_shape.size(); ++i)
    if (!std::isfinite(pwl_v_host[i])) return fail(c, MATEX_ERR_ARG, "non-finite PWL value");
  if (!zero_pattern_kept(c, pwl_v_host))
    return fail(c, MATEX_ERR_ARG,
                "the new currents are non-zero on a segment that setup skipped as identically "
                "zero; set up a new context");
  return MATEX_OK;
}

matex_status matex_set_sources(matex_ctx* c, const double* pwl_v_host) {
  if (!c) return MATEX_ERR_ARG;
  if (!pwl_v_host) return fail(c, MATEX_ERR_ARG, "pwl_v is NULL");
  if (c->opts.decompose == 1)
    return fail(c, MATEX_ERR_STATE, "decompose = 1 (ramps): set up a new context for new currents");
  matex_status cs = check_sources(c, pwl_v_host);
  if (cs != MATEX_OK) return cs;
  cudaMemcpyAsync(c->pwl_v_d, pwl_v_host, sizeof(double) * c->pwl_v_host_shape.size(),
                  cudaMemcpyHostToDevice, c->st);
  c->taped = false;
  return cuda_check(c, "set_sources");
}

matex_status matex_run_host(matex_ctx* c, const double* pwl_v_host, double* x_out_host,
                            matex_stats* stats) {
  if (!c) return MATEX_ERR_ARG;
  if (!x_out_host) return fail(c, MATEX_ERR_ARG, "x_out_host is NULL");
  if (pwl_v_host && c->opts.decompose == 1)
    return fail(c, MATEX_ERR_STATE, "decompose = 1 (ramps): set up a new context for new currents");
  const size_t bytes = sizeof(double) * (size_t)c->n_times * c->nrows_out;
  if (pwl_v_host) {
    matex_status cs = check_sources(c, pwl_v_host);
    if (cs != MATEX_OK) return cs;
    cudaMemcpyAsync(c->pwl_v_d, pwl_v_host, sizeof(double) * c->pwl_v_host_shape.size(),
                    cudaMemcpyHostToDevice, c->st);
  }
  // Page-locked host output: the final permutation kernel writes the voltages
  // straight into host memory through its device mapping (over NVLink-C2C on
  // Grace systems), so the device-to-host transfer is that kernel's stores.
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, x_out_host) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
      attr.devicePointer != nullptr) {
    matex_status s = run_device(c, static_cast<double*>(attr.devicePointer), stats);
    return s;
  }
  cudaGetLastError();
  if (!c->out_buf && !c->alloc(c->out_buf, (size_t)c->n_times * c->nrows_out))
    return fail(c, MATEX_ERR_OOM, "output buffer");
  matex_status s = run_device(c, c->out_buf, stats);
  if (s != MATEX_OK && s != MATEX_ERR_NOCONV) return s;
  if (cudaMemcpyAsync(x_out_host, c->out_buf, bytes, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return cuda_check(c, "run_host copy");
  return s;
}

matex_status matex_solve(matex_ctx* c, int32_t which, int32_t ncols, const double* b, double* x) {
  if (!c) return MATEX_ERR_ARG;
  if ((which != 0 && which != 1) || ncols < 0 || (ncols > 0 && (!b || !x)))
    return fail(c, MATEX_ERR_ARG, "bad solve arguments");
  const DevFactor& F = which == 0 ? c->fM : c->fG;
  const int64_t n = c->n;
  cudaMemsetAsync(c->d_count, 0, 4 * sizeof(int32_t), c->st);
  for (int32_t q0 = 0; q0 < ncols; q0 += c->ldy) {
    const int K = std::min<int>(c->ldy, ncols - q0);
    gather_cols(c->Y, c->ldy, K, b + (int64_t)q0 * n, n, nullptr, nullptr, c->perm, n, c->st);
    solve_cols(c, F, K);
    scatter_cols(c->Y, c->ldy, K, x + (int64_t)q0 * n, n, nullptr, c->perm, n, c->st);
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "solve sync");
  matex_status s = cuda_check(c, "solve");
  if (s != MATEX_OK) return s;
  int tmp = 0;
  return read_count(c, &tmp);
}

matex_status matex_solve_resident(matex_ctx* c, int32_t which, int32_t ncols, const double* b,
                                  double* x) {
  if (!c) return MATEX_ERR_ARG;
  if ((which != 0 && which != 1) || ncols < 0 || (ncols > 0 && (!b || !x)))
    return fail(c, MATEX_ERR_ARG, "bad solve arguments");
  if (!c->resident_ok)
    return fail(c, MATEX_ERR_STATE, "this context has no resident solve (grid too large, or "
                                    "krylov 2, tape, tail_eps or resident = 1 at setup)");
  resident_solve(which == 0 ? c->rM : c->rG, c->rplan, b, x, c->n, ncols, 1, c->n, c->perm, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "resident solve sync");
  return cuda_check(c, "resident solve");
}

matex_status matex_time_solve(matex_ctx* c, int32_t which, int32_t ncols, int32_t reps,
                              float* best_ms, float* mean_ms) {
  if (!c) return MATEX_ERR_ARG;
  if (which < 0 || which > 3 || ncols < 1 || ncols > c->ldy || reps < 1 || !best_ms)
    return fail(c, MATEX_ERR_ARG, "bad time_solve arguments (1 <= ncols <= column buffer width)");
  if (which >= 2 && !c->resident_ok)
    return fail(c, MATEX_ERR_STATE, "this context has no resident solve");
  const DevFactor& F = which % 2 == 0 ? c->fM : c->fG;
  // which 2, 3: the resident substitution, ncols columns of the buffer as n-vectors
  auto one = [&]() {
    if (which >= 2)
      resident_solve(which == 2 ? c->rM : c->rG, c->rplan, c->Y, c->Y, c->n, ncols, 1, c->n, nullptr,
                     c->st);
    else solve_cols(c, F, ncols);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_check(c, "time_solve events");
  }
  cudaMemsetAsync(c->d_count, 0, 4 * sizeof(int32_t), c->st);
  one();  // warm-up
  float best = 1e30f, sum = 0.f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, c->st);
    one();
    cudaEventRecord(e1, c->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
    sum += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  matex_status s = cuda_check(c, "time_solve");
  if (s != MATEX_OK) return s;
  int tmp = 0;
  if ((s = read_count(c, &tmp)) != MATEX_OK) return s;
  *best_ms = best;
  if (mean_ms) *mean_ms = sum / (float)reps;
  return MATEX_OK;
}

matex_status matex_expm(matex_ctx* c, int32_t batch, int32_t m, const double* A, const double* h,
                        double* E) {
  if (!c) return MATEX_ERR_ARG;
  if (batch < 0 || m < 1 || m > kMaxM || (batch > 0 && (!A || !h || !E)))
    return fail(c, MATEX_ERR_ARG, "bad expm arguments");
  if (batch == 0) return MATEX_OK;
  expm_batch(batch, m, A, h, E, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "expm sync");
  return cuda_check(c, "expm");
}

matex_status matex_get_m(matex_ctx* c, int32_t* m_host, int64_t cap, int64_t* count) {
  if (!c) return MATEX_ERR_ARG;
  if (count) *count = c->n_segments;
  if (m_host && cap > 0 && c->n_segments > 0) {
    const int64_t k = std::min(cap, c->n_segments);
    if (cudaMemcpy(m_host, c->m_rec, sizeof(int32_t) * k, cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_check(c, "get_m");
  }
  return MATEX_OK;
}

matex_status matex_get_sizes(matex_ctx* c, int32_t* n_times, int32_t* n_rows, int64_t* n_segments) {
  if (!c) return MATEX_ERR_ARG;
  if (n_times) *n_times = c->n_times;
  if (n_rows) *n_rows = c->nrows_out;
  if (n_segments) *n_segments = c->n_segments;
  return MATEX_OK;
}

matex_status matex_set_batching(matex_ctx* c, int32_t one_group_at_a_time) {
  if (c && one_group_at_a_time && c->batches.size() > 1)
    return fail(c, MATEX_ERR_STATE, "one group at a time is not available for batched ramp columns");
  if (!c) return MATEX_ERR_ARG;
  const bool serial = one_group_at_a_time != 0;
  if (serial != c->serial) drop_graph(c);  // another launch sequence
  c->serial = serial;
  return MATEX_OK;
}

matex_status matex_debug_inject_wait(matex_ctx* c, int32_t on) {
  if (!c) return MATEX_ERR_ARG;
  c->inject_wait = on != 0;
  return MATEX_OK;
}

matex_status matex_get_autotune(matex_ctx* c, int32_t* ncols, int32_t* mode, float* ms,
                               int32_t cap, int32_t* count) {
  if (!c) return MATEX_ERR_ARG;
  const int k = (int)c->tune_reps.size();
  if (count) *count = k;
  for (int i = 0; i < std::min(cap, k); ++i) {
    if (ncols) ncols[i] = c->tune_reps[i];
    if (mode) mode[i] = c->tune_modes[i];
    if (ms) {
      const bool have = 2 * (size_t)i + 1 < c->tune_ms.size();
      ms[2 * i] = have ? c->tune_ms[2 * i] : -1.f;
      ms[2 * i + 1] = have ? c->tune_ms[2 * i + 1] : -1.f;
    }
  }
  return MATEX_OK;
}

matex_status matex_get_level_blocks(matex_ctx* c, int32_t* kb_fwd, int32_t* kb_bwd, float* ms,
                                    int32_t cap, int32_t* nlev) {
  if (!c) return MATEX_ERR_ARG;
  if (!nlev || cap < 0 || (cap > 0 && (!kb_fwd || !kb_bwd))) return fail(c, MATEX_ERR_ARG, "NULL argument");
  const int L = (int)c->levels.size();
  *nlev = L;
  for (int l = 0; l < L && l < cap; ++l) {
    kb_fwd[l] = c->levels[l].kbf;
    kb_bwd[l] = c->levels[l].kbb;
    if (ms) {
      const bool tuned = c->level_tune_ms.size() == (size_t)(2 * L);
      ms[2 * l] = tuned ? c->level_tune_ms[2 * l] : -1.f;
      ms[2 * l + 1] = tuned ? c->level_tune_ms[2 * l + 1] : -1.f;
    }
  }
  return MATEX_OK;
}

matex_status matex_set_profiling(matex_ctx* c, int32_t on) {
  if (!c) return MATEX_ERR_ARG;
  c->prof_on = on != 0;
  if (c->prof_on) {
    std::memset(&c->prof, 0, sizeof(c->prof));
    c->pend.clear();
    c->ev_used = 0;
  }
  return MATEX_OK;
}

matex_status matex_get_profile(matex_ctx* c, matex_profile* out) {
  if (!c || !out) return MATEX_ERR_ARG;
  *out = c->prof;
  return MATEX_OK;
}

matex_status matex_get_setup_stats(matex_ctx* c, matex_stats* stats) {
  if (!c) return MATEX_ERR_ARG;
  if (stats) *stats = c->setup_stats;
  return MATEX_OK;
}

}  // extern "C"

extern "C" matex_status matex_host_factor_solve(int64_t n, const int64_t* rowptr, const int32_t* col,
                                                const double* val, const double* dshift,
                                                double alpha, int32_t max_width, int32_t ncols,
                                                const double* b, double* x, int64_t* info) {
  g_setup_err.clear();
  if (n <= 0 || !rowptr || !col || !val || ncols < 0 || (ncols > 0 && (!b || !x))) {
    g_setup_err = "bad arguments";
    return MATEX_ERR_ARG;
  }
  CsrSym A{n, rowptr, col, val};
  std::vector<int32_t> nd;
  Symbolic S;
  std::string e = nested_dissection(A, nd);
  if (e.empty()) e = symbolic_analysis(A, nd, max_width > 0 ? max_width : 128, S);
  if (!e.empty()) { g_setup_err = e; return MATEX_ERR_ARG; }
  Numeric F;
  e = numeric_ldlt(A, dshift, alpha, S, F);
  if (!e.empty()) { g_setup_err = e; return MATEX_ERR_NOT_SPD; }
  int64_t maxw = 0;
  for (int32_t s = 0; s < S.nsup; ++s) maxw = std::max<int64_t>(maxw, S.sup_first[s + 1] - S.sup_first[s]);
  if (info) {
    info[0] = S.nnz_L;
    info[1] = S.nsup;
    info[2] = (int64_t)S.level_ptr.size() - 1;
    info[3] = maxw;
    info[4] = S.nnz_L_exact;
  }
  std::vector<double> y(n), tmp;
  for (int32_t q = 0; q < ncols; ++q) {
    for (int64_t k = 0; k < n; ++k) y[k] = b[(int64_t)q * n + S.perm[k]];
    // forward, supernodes in level order (as the GPU launches them): P_s b_s
    for (size_t li = 0; li < S.level_sups.size(); ++li) {
      const int32_t s = S.level_sups[li];
      const int32_t f = S.sup_first[s], w = S.sup_first[s + 1] - f;
      const int64_t rp = S.sup_rowptr[s];
      const int32_t ld = (int32_t)(S.sup_rowptr[s + 1] - rp);
      const double* P = &F.pan_cm[S.pan_off[s]];
      tmp.assign(ld, 0.0);
      for (int32_t j = 0; j < w; ++j)
        for (int32_t i = 0; i < ld; ++i) tmp[i] += P[(int64_t)j * ld + i] * y[f + j];
      for (int32_t i = 0; i < w; ++i) y[f + i] = tmp[i];
      for (int32_t i = w; i < ld; ++i) y[S.sup_rows[rp + i]] -= tmp[i];
    }
    // backward, reverse level order: P_s^T [D^{-1} y_s; -x_R]
    for (size_t li = S.level_sups.size(); li-- > 0;) {
      const int32_t s = S.level_sups[li];
      const int32_t f = S.sup_first[s], w = S.sup_first[s + 1] - f;
      const int64_t rp = S.sup_rowptr[s];
      const int32_t ld = (int32_t)(S.sup_rowptr[s + 1] - rp);
      const double* P = &F.pan_rm[S.pan_off[s]];
      tmp.assign(ld, 0.0);
      for (int32_t i = 0; i < ld; ++i) {
        const double v = y[S.sup_rows[rp + i]];
        tmp[i] = i < w ? v * F.dinv[f + i] : -v;
      }
      for (int32_t j = 0; j < w; ++j) {
        double acc = 0.0;
        for (int32_t i = 0; i < ld; ++i) acc += P[(int64_t)i * w + j] * tmp[i];
        y[f + j] = acc;
      }
    }
    for (int64_t k = 0; k < n; ++k) x[(int64_t)q * n + S.perm[k]] = y[k];
  }
  return MATEX_OK;
}

// Host-only check of the single-column kernels' plan: builds it for G (the
// setup's ordering and symbolic analysis) and walks every warp's lanes the
// way the kernels find their rows (prefix of the row counts of the warp's
// first 32 records, five-step search), checking that each lane lands in a
// record of its level and group size, inside the record, and that every row
// (forward) and column (backward) of every supernode is taken by exactly one
// group of lanes.
extern "C" matex_status matex_host_single_column_plan(int64_t n, const int64_t* rowptr,
                                                      const int32_t* col, const double* val,
                                                      int32_t max_width, int64_t* info) {
  g_setup_err.clear();
  if (n <= 0 || !rowptr || !col || !val) {
    g_setup_err = "bad arguments";
    return MATEX_ERR_ARG;
  }
  CsrSym A{n, rowptr, col, val};
  std::vector<int32_t> nd;
  Symbolic S;
  std::string e = nested_dissection(A, nd);
  if (e.empty()) e = symbolic_analysis(A, nd, max_width > 0 ? max_width : 1024, S);
  if (!e.empty()) { g_setup_err = e; return MATEX_ERR_ARG; }
  std::vector<K1Sup> recs[2];
  std::vector<K1Warp> warps[2];
  std::vector<int32_t> off[2];
  build_k1_plan(S, recs, warps, off);
  const int nlev = (int)S.level_ptr.size() - 1;
  const int nsup = S.nsup;
  int64_t errors = 0, units[2] = {0, 0};
  for (int dir = 0; dir < 2; ++dir) {
    const bool fwd = dir == 0;
    const std::vector<K1Sup>& R = recs[dir];
    auto count_of = [&](int r) { return fwd ? R[r].ld : R[r].w; };
    auto lg_of = [&](int r) {
      const int len = fwd ? R[r].w : R[r].ld;
      int lg = 0;
      while (lg < 5 && 16 * (1 << lg) < len) ++lg;
      return lg;
    };
    std::vector<int64_t> first(R.size() + 1, 0);
    for (size_t r = 0; r < R.size(); ++r) first[r + 1] = first[r] + count_of((int)r);
    std::vector<int32_t> taken(first.back(), 0);
    for (int l = 0; l < nlev; ++l) {
      const int r0 = S.level_ptr[l], r1 = S.level_ptr[l + 1];
      for (int wi = off[dir][l]; wi < off[dir][l + 1]; ++wi) {
        const K1Warp wp = warps[dir][wi];
        int pre[32];
        for (int j = 0; j < 32; ++j) {
          const int r = wp.k0 + j;
          pre[j] = (j ? pre[j - 1] : 0) + (r < nsup ? count_of(r) : 0);
        }
        const int G = 1 << wp.lg;
        if (wp.nslot < 1 || wp.nslot > 32 / G) ++errors;
        for (int lane = 0; lane < 32; lane += G) {
          const int slot = lane >> wp.lg;
          if (slot >= wp.nslot) continue;
          const int row = wp.i0 + slot;
          int m = 0;
          for (int b = 16; b > 0; b >>= 1)
            if (pre[m + b - 1] <= row) m += b;
          const int rec = wp.k0 + m;
          const int i = row - (m > 0 ? pre[m - 1] : 0);
          if (m >= 32 || rec < r0 || rec >= r1 || lg_of(rec) != wp.lg || i < 0 ||
              i >= count_of(rec)) {
            ++errors;
            continue;
          }
          ++taken[first[rec] + i];
        }
      }
    }
    for (int32_t t : taken) errors += t != 1;
    units[dir] = first.back();
  }
  if (info) {
    info[0] = nlev;
    info[1] = off[0][nlev];
    info[2] = off[1][nlev];
    info[3] = units[0];
    info[4] = units[1];
    info[5] = errors;
  }
  if (errors) {
    g_setup_err = "single-column plan: " + std::to_string(errors) + " mapping errors";
    return MATEX_ERR_STATE;
  }
  return MATEX_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free solve.  Code that must not touch the CUDA allocator (it runs
// where cudaMalloc is forbidden or would deadlock, e.g. inside another
// library's allocator callback, or in a process whose memory pool is owned by
// someone else) can still solve with a context's factors through
// matex_solve_noalloc: it uses no context work buffer and allocates nothing,
// taking its right-hand-side buffers and dependency counters from the static
// device array below.  Every GPU that loads the library holds this array
// until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = 16u << 20;      // 16 MiB per device
constexpr size_t kNoAllocCounterBytes = 2u << 20;  // first 2 MiB: ticket, error flag, counters
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static array on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
matex_status noalloc_scratch(int dev, void** out, std::string& err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal out of range";
    return MATEX_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return MATEX_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MATEX_OK;
}

}  // namespace

extern "C" matex_status matex_solve_noalloc(matex_ctx* c, int32_t which, int32_t ncols,
                                            const double* b, double* x) {
  if (!c) return MATEX_ERR_ARG;
  if ((which != 0 && which != 1) || ncols < 0 || (ncols > 0 && (!b || !x)))
    return fail(c, MATEX_ERR_ARG, "bad solve arguments");
  if (ncols == 0) return MATEX_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return fail(c, MATEX_ERR_ARG, "the context's device must be current");
  const int64_t n = c->n;
  const int32_t nsup = c->S.nsup;
  // counters: ticket (8 B), error flag (8 B), fdone, bdone, fpend (nsup ints each)
  const size_t counter_need = 16 + 3 * sizeof(int) * (size_t)nsup;
  if (counter_need > kNoAllocCounterBytes)
    return fail(c, MATEX_ERR_ARG, "matex_solve_noalloc: the factor has more than " +
                                      std::to_string((kNoAllocCounterBytes - 16) / 12) +
                                      " supernodes (its static scratch limit)");
  const size_t rhs_doubles = (kNoAllocBytes - kNoAllocCounterBytes) / sizeof(double);
  // Leading dimension of a chunk of kc columns.  Every solve kernel works on
  // column blocks of KB columns, KB a power of two up to kMaxColBlock, halved
  // while KB / 2 >= kc (run_level and the persistent schedule): the blocks of
  // a chunk then end at kc rounded up to KB, which ld_for(kc) covers.
  static_assert(kMaxColBlock <= 8 && (kMaxColBlock & (kMaxColBlock - 1)) == 0,
                "ld_for holds the column blocks only for power-of-two blocks up to 8");
  auto ld_for = [](int kc) { return kc <= 1 ? 1 : kc <= 2 ? 2 : kc <= 4 ? 4 : (kc + 7) & ~7; };
  // widest column chunk whose Y and Y2 fit the static scratch
  int kc = std::min<int>(ncols, c->ldy);
  while (kc > 1 && 2 * (size_t)n * ld_for(kc) > rhs_doubles) kc = kc > 8 ? ((kc - 1) & ~7) : kc - 1;
  if (2 * (size_t)n * ld_for(kc) > rhs_doubles)
    return fail(c, MATEX_ERR_ARG, "matex_solve_noalloc: n = " + std::to_string(n) +
                                      " exceeds the static scratch (at most " +
                                      std::to_string(rhs_doubles / 2) + " nodes)");
  void* base = nullptr;
  matex_status s = noalloc_scratch(dev, &base, c->err);
  if (s != MATEX_OK) return s;
  unsigned char* bytes = static_cast<unsigned char*>(base);
  unsigned long long* ticket = reinterpret_cast<unsigned long long*>(bytes);
  int* err = reinterpret_cast<int*>(bytes + 8);
  int* fdone = reinterpret_cast<int*>(bytes + 16);
  int* bdone = fdone + nsup;
  int* fpend = bdone + nsup;
  double* Y = reinterpret_cast<double*>(bytes + kNoAllocCounterBytes);
  const DevFactor& F = which == 0 ? c->fM : c->fG;
  const int nlev = (int)c->levels.size();
  cudaStream_t st = c->st;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  for (int32_t q0 = 0; q0 < ncols; q0 += kc) {
    const int K = std::min<int>(kc, ncols - q0);
    const int ldy = ld_for(K);
    double* Y2 = Y + (size_t)n * ldy;
    gather_cols(Y, ldy, K, b + (int64_t)q0 * n, n, nullptr, nullptr, c->perm, n, st);
    int mode = c->opts.solve_mode;
    if (mode == 2) mode = c->mode_by_ncols.empty() ? 0 : c->mode_by_ncols[std::min(K, c->ldy)];
    if (mode == 1) {
      // one launch per tree level: no counters, only the two column buffers
      solve_inplace(F, c->levels.data(), nlev, Y, Y2, ldy, K, st);
      scatter_cols(Y, ldy, K, x + (int64_t)q0 * n, n, nullptr, c->perm, n, st);
      continue;
    }
    PersistSched ps;
    ps.lev = c->plev_d + (size_t)(K - 1) * nlev;
    ps.nlev = nlev;
    ps.nf_total = c->pf_total[K];
    ps.nb_total = c->pb_total[K];
    ps.ticket = ticket;
    ps.fdone = fdone;
    ps.bdone = bdone;
    ps.fpend = fpend;
    ps.err = err;
    ps.sup_level = c->sup_level_d;
    ps.nft = c->nft_d;
    ps.nbt = c->nbt_d;
    // everything a solve counts up from starts at zero; fpend starts at the child counts
    cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(fdone, 0, 2 * sizeof(int) * (size_t)nsup, st);
    cudaMemcpyAsync(fpend, c->fpend_init, sizeof(int) * nsup, cudaMemcpyDeviceToDevice, st);
    persistent_solve(F, ps, c->pgrid, c->psmem, Y, Y2, ldy, st);
    scatter_cols(Y, ldy, K, x + (int64_t)q0 * n, n, nullptr, c->perm, n, st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "solve_noalloc sync");
  if ((s = cuda_check(c, "solve_noalloc")) != MATEX_OK) return s;
  int flag = 0;
  if (cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(c, "solve_noalloc flag");
  if (flag) return fail(c, MATEX_ERR_TIMEOUT, "a bounded wait of the persistent solve expired");
  return MATEX_OK;
}

// ---------------------------------------------------------------------------
// Fixed-step trapezoidal integration (Eq. 2), the paper's comparison method,
// on the same batched solves.
// ---------------------------------------------------------------------------
namespace {

// Factor C + h/2 G on the host with the context's symbolic structure and
// upload it (panels allocated once, rewritten when h changes); G in CSR in
// the permuted order on first use.
matex_status tr_prepare(matex_ctx* c, double h) {
  const int64_t n = c->n;
  if (!ensure_g_csr(c) || (!c->trX && (!c->alloc(c->trX, n) || !c->alloc(c->trB0, n) ||
                                        !c->alloc(c->trB1, n))))
    return fail(c, MATEX_ERR_OOM, "trapezoidal buffers");
  if (c->tr_h == h) return MATEX_OK;
  const double t0 = now_ms();
  CsrSym A{n, c->g_rowptr_h.data(), c->g_col_h.data(), c->g_val_h.data()};
  Numeric NT;
  const std::string e = numeric_ldlt(A, c->c_host.data(), 0.5 * h, c->S, NT);
  if (!e.empty()) return fail(c, MATEX_ERR_NOT_SPD, e);
  if (!c->fT.dinv) {
    double *d, *pc, *pr;
    if (!c->alloc(d, NT.dinv.size()) || !c->alloc(pc, NT.pan_cm.size()) || !c->alloc(pr, NT.pan_rm.size()))
      return fail(c, MATEX_ERR_OOM, "trapezoidal factor");
    c->fT = c->fM;
    c->fT.dinv = d;
    c->fT.pan_cm = pc;
    c->fT.pan_rm = pr;
    c->fT.abort = nullptr;
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess ||
      cudaMemcpy(const_cast<double*>(c->fT.dinv), NT.dinv.data(), sizeof(double) * NT.dinv.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(const_cast<double*>(c->fT.pan_cm), NT.pan_cm.data(), sizeof(double) * NT.pan_cm.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(const_cast<double*>(c->fT.pan_rm), NT.pan_rm.data(), sizeof(double) * NT.pan_rm.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check(c, "trapezoidal factor upload");
  c->tr_h = h;
  c->tr_factor_ms = now_ms() - t0;
  if (c->tr_exec) cudaGraphExecDestroy(c->tr_exec);
  c->tr_exec = nullptr;
  return MATEX_OK;
}

// The whole integration on c->st: DC start x_0 = G^{-1} b(0), then N*substeps
// steps; the state at every output time goes to Xp.
void tr_pass(matex_ctx* c, int substeps, double h) {
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  const double* dc = c->opts.include_dc ? c->dc_perm : nullptr;
  double* bp = c->trB0;
  double* bn = c->trB1;
  tr_input(bp, dc, c->src, c->n_src, 0.0, n, st);
  gather_cols(c->Y, c->ldy, 1, bp, 0, nullptr, nullptr, nullptr, n, st);
  solve_cols(c, c->fG, 1);
  tr_store(c->trX, c->Y, c->ldy, c->Xp, 0, n, st);
  const int64_t steps = (int64_t)(c->n_times - 1) * substeps;
  for (int64_t k = 1; k <= steps; ++k) {
    tr_input(bn, dc, c->src, c->n_src, (double)k * h, n, st);
    tr_rhs(c->Y, c->ldy, c->trX, c->trG_rowptr, c->trG_col, c->trG_val, c->c_perm, 0.5 * h, bp, bn,
           n, st);
    solve_cols(c, c->fT, 1);
    tr_store(c->trX, c->Y, c->ldy, c->Xp, k % substeps == 0 ? k / substeps : -1, n, st);
    std::swap(bp, bn);
  }
}

}  // namespace

extern "C" matex_status matex_tr_run(matex_ctx* c, int32_t substeps, double* x_out, double* ms_out) {
  if (!c) return MATEX_ERR_ARG;
  if (substeps < 1 || !x_out) return fail(c, MATEX_ERR_ARG, "substeps must be >= 1 and x_out set");
  const double h = c->dt_out / substeps;
  matex_status s = tr_prepare(c, h);
  if (s != MATEX_OK) return s;
  if (c->tr_substeps != substeps && c->tr_exec) {
    cudaGraphExecDestroy(c->tr_exec);
    c->tr_exec = nullptr;
  }
  // record the loop once (about 40 launches per step, no host decision in it)
  if (!c->tr_exec && !c->inject_wait) {
    if (!c->gst && cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->gst = nullptr;
    }
    if (c->gst) {
      cudaStream_t user = c->st;
      c->st = c->gst;
      cudaGraph_t g = nullptr;
      bool ok = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        tr_pass(c, substeps, h);
        ok = cudaStreamEndCapture(c->gst, &g) == cudaSuccess && g != nullptr;
      }
      c->st = user;
      if (ok) ok = cudaGraphInstantiate(&c->tr_exec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      if (!ok) c->tr_exec = nullptr;
      cudaGetLastError();
      c->tr_substeps = substeps;
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(c->d_count, 0, 4 * sizeof(int32_t), c->st);
  cudaEventRecord(e0, c->st);
  if (c->tr_exec) cudaGraphLaunch(c->tr_exec, c->st);
  else tr_pass(c, substeps, h);
  cudaEventRecord(e1, c->st);
  permute_out(x_out, c->Xp, c->out_map, c->nrows_out, c->n, c->n_times, c->st);
  const bool ok = cudaStreamSynchronize(c->st) == cudaSuccess;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return cuda_check(c, "trapezoidal run");
  if ((s = cuda_check(c, "trapezoidal run")) != MATEX_OK) return s;
  int tmp = 0;
  if ((s = read_count(c, &tmp)) != MATEX_OK) return s;
  if (ms_out) *ms_out = ms;
  return MATEX_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent contexts (grids of different sizes) as one CUDA
// graph launch: a start event, then one child-graph branch per context (its
// recorded run), each followed by its own end event.  The branches share no
// edges, so the GPU runs them concurrently.
// ---------------------------------------------------------------------------
struct matex_batch {
  std::vector<matex_ctx*> ctxs;
  std::vector<int64_t> gens;    // recording generation of each context in the built graph
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // [0] batch start, [1 + i] end of context i's branch
  cudaStream_t st = nullptr;
  std::string err;
  ~matex_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

namespace {

matex_status batch_fail(matex_batch* b, matex_status s, const std::string& m) {
  b->err = m;
  return s;
}

// A plain run of context c into its own device buffer, which records its graph.
matex_status batch_record(matex_batch* b, matex_ctx* c) {
  if (!c->out_buf && !c->alloc(c->out_buf, (size_t)c->n_times * c->nrows_out))
    return batch_fail(b, MATEX_ERR_OOM, "output buffer");
  matex_status s = run_device(c, c->out_buf, nullptr);
  if (s != MATEX_OK && s != MATEX_ERR_NOCONV) return batch_fail(b, s, c->err);
  if (!c->graph) return batch_fail(b, MATEX_ERR_CUDA, "a context's run could not be recorded as a graph");
  return MATEX_OK;
}

matex_status batch_build(matex_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaGraph_t parent = nullptr;
  if (cudaGraphCreate(&parent, 0) != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(b, MATEX_ERR_CUDA, "cudaGraphCreate failed");
  }
  cudaGraphNode_t start;
  bool ok = cudaGraphAddEventRecordNode(&start, parent, nullptr, 0, b->ev[0]) == cudaSuccess;
  for (size_t i = 0; ok && i < b->ctxs.size(); ++i) {
    cudaGraphNode_t child, end;
    ok = cudaGraphAddChildGraphNode(&child, parent, &start, 1, b->ctxs[i]->graph) == cudaSuccess &&
         cudaGraphAddEventRecordNode(&end, parent, &child, 1, b->ev[1 + i]) == cudaSuccess;
    b->gens[i] = b->ctxs[i]->graph_gen;
  }
  if (ok) ok = cudaGraphInstantiate(&b->exec, parent, 0) == cudaSuccess;
  cudaGraphDestroy(parent);
  if (!ok) {
    b->exec = nullptr;
    return batch_fail(b, MATEX_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(cudaGetLastError()));
  }
  return MATEX_OK;
}

}  // namespace

extern "C" {

matex_status matex_batch_create(matex_batch** out, matex_ctx* const* ctxs, int32_t count) {
  if (!out) return MATEX_ERR_ARG;
  *out = nullptr;
  if (!ctxs || count <= 0) return MATEX_ERR_ARG;
  for (int32_t i = 0; i < count; ++i) {
    if (!ctxs[i] || !ctxs[i]->opts.graph) return MATEX_ERR_ARG;
    if (ctxs[i]->device != ctxs[0]->device) return MATEX_ERR_ARG;
    for (int32_t k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return MATEX_ERR_ARG;
  }
  matex_batch* b = new (std::nothrow) matex_batch();
  if (!b) return MATEX_ERR_OOM;
  b->ctxs.assign(ctxs, ctxs + count);
  b->gens.assign(count, -1);
  b->st = ctxs[0]->st;
  for (int32_t i = 0; i <= count; ++i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return MATEX_ERR_CUDA;
    }
    b->ev.push_back(e);
  }
  matex_status s = MATEX_OK;
  for (matex_ctx* c : b->ctxs)
    if (!c->graph && (s = batch_record(b, c)) != MATEX_OK) break;
  if (s == MATEX_OK) s = batch_build(b);
  if (s != MATEX_OK) {
    g_setup_err = b->err;
    delete b;
    return s;
  }
  *out = b;
  return MATEX_OK;
}

matex_status matex_batch_run(matex_batch* b, double* const* x_outs, matex_stats* stats, float* grid_ms) {
  if (!b) return MATEX_ERR_ARG;
  const size_t nb = b->ctxs.size();
  if (!x_outs) return batch_fail(b, MATEX_ERR_ARG, "x_outs is NULL");
  for (size_t i = 0; i < nb; ++i)
    if (!x_outs[i]) return batch_fail(b, MATEX_ERR_ARG, "an output pointer is NULL");
  // contexts re-recorded (or dropped) since the batch graph was built
  bool rebuild = !b->exec;
  matex_status s;
  for (size_t i = 0; i < nb; ++i) {
    matex_ctx* c = b->ctxs[i];
    if (c->prof_on || c->inject_wait)
      return batch_fail(b, MATEX_ERR_STATE, "profiling or wait injection is on for a context");
    if (!c->graph && (s = batch_record(b, c)) != MATEX_OK) return s;
    if (c->graph_gen != b->gens[i]) rebuild = true;
  }
  if (rebuild && (s = batch_build(b)) != MATEX_OK) return s;
  // work queued earlier on the contexts' own streams comes first
  for (matex_ctx* c : b->ctxs)
    if (c->st != b->st && cudaStreamSynchronize(c->st) != cudaSuccess)
      return batch_fail(b, MATEX_ERR_CUDA, "context stream sync failed");
  const double t0 = now_ms();
  if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess)
    return batch_fail(b, MATEX_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(cudaGetLastError()));
  for (size_t i = 0; i < nb; ++i) {
    matex_ctx* c = b->ctxs[i];
    permute_out(x_outs[i], c->Xp, c->out_map, c->nrows_out, c->n, c->n_times, b->st);
    cudaMemcpyAsync(c->h_count, c->d_count, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, b->st);
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return batch_fail(b, MATEX_ERR_CUDA, "batch run failed");
  matex_status worst = MATEX_OK;
  for (size_t i = 0; i < nb; ++i) {
    matex_ctx* c = b->ctxs[i];
    if (grid_ms) {
      grid_ms[i] = 0.f;
      cudaEventElapsedTime(&grid_ms[i], b->ev[0], b->ev[1 + i]);
    }
    if (c->h_count[1] != 0)
      return batch_fail(b, MATEX_ERR_TIMEOUT, "a bounded wait of the persistent solve expired");
    matex_stats* si = stats ? stats + i : nullptr;
    if (c->h_count[2] != 0) {
      // this grid's counts diverged from its recording: redo it plainly
      drop_graph(c);
      s = run_device(c, x_outs[i], si);
    } else {
      s = finish_run(c, c->graph_counts, t0, true, si);
    }
    if (s == MATEX_ERR_NOCONV) worst = s;
    else if (s != MATEX_OK) return batch_fail(b, s, c->err);
  }
  return worst;
}

const char* matex_batch_last_error(const matex_batch* b) { return b ? b->err.c_str() : ""; }

void matex_batch_destroy(matex_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  delete b;
}

}  // extern "C"
