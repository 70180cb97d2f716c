// Launch wrappers of the R-MATEX CUDA kernels (internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace matex {

constexpr int kMaxM = 20;      // largest Krylov dimension
constexpr int kMaxB = kMaxM + 1;
// coefficient row per (column, output): y_0..y_{m-1} in slots 0..m-1 and the
// step h = t_o - l_j of the -P term in slot kMaxM
constexpr int kCoefLd = kMaxM + 1;

// Device view of one factor on the shared structure: D^{-1} and the solve
// panels P_s = [L_ss^{-1}; L_Rs L_ss^{-1}] ((w+r) x w), column- and row-major.
struct DevFactor {
  const int32_t* sup_first;
  const int32_t* sup_parent;
  const int64_t* sup_rowptr;
  const int32_t* sup_rows;
  const int64_t* pan_off;
  const double* dinv;
  const double* pan_cm;
  const double* pan_rm;
  const int32_t* pack;   // supernode lists of packed tasks
  const int32_t* pack_a; // per pack entry: panel rows (sum of w + r) of the task's earlier entries
  const int32_t* pack_b; // per pack entry: panel columns (sum of w) of the task's earlier entries
  const int32_t* abort = nullptr;  // device flag or null: when set before a launch, its CTAs exit at once
                         // (a graph replay whose counts diverged; its result is discarded)
};

constexpr int kMaxColBlock = 8;  // largest column block KB of the solve kernels (a power of two)
constexpr int kRowBlock = 32;  // panel rows (forward) / columns (backward) per task
constexpr int kPackRows = 128; // rows (forward) / columns (backward) of a packed task
constexpr int kPackMax = 64;   // supernodes per packed task
// Flag in a packed task's count: one thread per panel row (forward) or column
// (backward) instead of warp-wide (row or column, right-hand side) chunks.
constexpr int kPackRowwise = 1 << 16;
// A task is int2 {s, first row/column} for one supernode, or, for many small
// supernodes of one level, int2 {-1 - e, count}: pack[e .. e+count) lists them
// and the task runs one thread per panel row (forward) / column (backward).

// One tree level of the supernodal solve.  A task is (supernode, block of 32
// panel rows) in the forward direction and (supernode, block of 32 panel
// columns) in the backward one; each task runs once per column block.
struct LevelPlan {
  const int2* ftasks;    // device, {supernode, first panel row}
  const int2* btasks;    // device, {supernode, first panel column}
  int32_t nf, nb;
  int32_t max_w;         // widest supernode in the level
  int32_t max_wr;        // largest w + r in the level
  int32_t kb;            // column block: 1, 2, 4 or 8 (occupancy rule; persistent schedule)
  int32_t kbf, kbb;      // column blocks of the level launches, forward and backward
                         // (set by the setup-time tuner, else kb)
  int32_t split_w;       // widest supernode with split (non-packed) tasks, 0 if none: the
                         // longest reduction of a forward task
  int32_t split_ld;      // largest w + r of those: the longest reduction of a backward task
};

// Scratch of the chunked reduction.  A split task whose level would leave
// the GPU mostly idle (few tasks x column blocks) runs as `nchunk` CTAs, each
// over one slice of the task's reduction (panel columns forward, panel rows
// backward).  Their partial sums of the rows that need a complete sum (the
// diagonal block forward, every output backward) go to `part`; the CTA that
// arrives last, counted in `cnt` (zero between launches: that CTA resets
// it), adds them in chunk order and writes the result.  No CTA waits on
// another.  Rows below the diagonal block take each chunk's partial by an
// atomic subtraction, like the unchunked forward.
struct SplitScratch {
  double* part = nullptr;  // [kSplitSlots * 2][kRowBlock][kMaxColBlock]
  int* cnt = nullptr;      // [kSplitSlots]
};
constexpr int kSplitTarget = 4 * 152;  // CTAs a level launch should reach (4 per SM)
constexpr int kSplitSlots = kSplitTarget;
constexpr int kSplitMaxChunks = 32;
constexpr int kSplitMinWidth = 32;     // columns (rows) of one chunk at least
void set_solve_smem_limit(int bytes);

// Persistent (one launch per solve) schedule for a given column count.
// A ticket covers `fbatch` (forward) or `bbatch` (backward) consecutive tasks
// of one level, run in order by the CTA that draws it: large levels of small
// tasks draw fewer tickets, small levels keep one task per ticket.
struct PersistLevel {
  const int2* ftasks;
  const int2* btasks;
  int32_t nf, nb;       // tasks of the level in each direction (before column blocks)
  int32_t kb, ncb;      // column block and number of column blocks
  int32_t fbatch, bbatch;
  long long fbase;      // first forward ticket of the level
  long long bbase;      // first backward ticket of the level (backward counts top-down)
};
struct PersistSched {
  const PersistLevel* lev;
  int nlev;
  long long nf_total, nb_total;
  unsigned long long* ticket;
  int* fdone;            // [nsup] completed forward tasks
  int* bdone;            // [nsup] completed backward tasks
  int* fpend;            // [nsup] children whose forward tasks are not all done
  int* err;              // set on a wait timeout
  const int32_t* sup_level;
  const int32_t* nft;    // [nsup] forward row blocks per supernode
  const int32_t* nbt;    // [nsup] backward column blocks per supernode
};
void persistent_solve(const DevFactor& F, const PersistSched& ps, int grid, size_t smem,
                      double* Y, double* Y2, int ldy, cudaStream_t st);
int persistent_blocks_per_sm(size_t smem);
// Loads every kernel a solve can launch (level kernels of every column block,
// the persistent kernel, the gathers and scatters) on the current device, so
// that a later solve triggers no lazy module loading (which allocates device
// memory for the code).  Returns false on a CUDA error.
bool preload_solve_kernels();
// Device time (best of reps after a warm-up, CUDA events on st) of one level
// launch with column block kb for ncols right-hand sides; -1 on an error.
float time_level(bool fwd, const DevFactor& F, const LevelPlan& L, int kb, double* Y, double* Y2,
                 int ldy, int ncols, cudaStream_t st, const SplitScratch* split, int reps);
constexpr int kSolveSmemTune = 100 * 1024;  // largest staging buffer a tuned column block may use
// adds one to *p on the stream (failure-injection hook of the tests)
void bump_counter(int* p, cudaStream_t st);

// Y is node-major [n][ldy] (ldy >= ncols, multiple of 8); solves in place,
// using Y2 (same shape) for the intermediate forward result.
// Returns the number of kernels launched.
int solve_inplace(const DevFactor& F, const LevelPlan* levels, int nlev, double* Y, double* Y2,
                  int ldy, int ncols, cudaStream_t st, const SplitScratch* split = nullptr);

// Y[i][q] = (scale ? scale[i] : 1) * src[cols[q]*stride + rowmap[i]]
// (cols == null: q; rowmap == null: i)
void gather_cols(double* Y, int ldy, int ncols, const double* src, int64_t stride,
                 const int32_t* cols, const double* scale, const int32_t* rowmap, int64_t n,
                 cudaStream_t st);
// dst[cols[q]*stride + rowmap[i]] = Y[i][q]
void scatter_cols(const double* Y, int ldy, int ncols, double* dst, int64_t stride,
                  const int32_t* cols, const int32_t* rowmap, int64_t n, cudaStream_t st);

// Per-column metadata of one segment round (device arrays, length K).
struct RoundCols {
  const int32_t* group;    // group of the column
  const int32_t* vslot;    // slot of its Krylov basis: the group, or the segment record
                           // when every segment keeps its basis (adjoint tape)
  const int32_t* seg;      // segment index inside the group
  const double* l0;        // segment start
  const double* len;       // segment length L
  const double* hfirst;    // offset of the first output in the segment (L if none)
  const double* lprev;     // length of the group's previous segment (0 for the first)
  const int32_t* obeg;     // first output index in the segment
  const int32_t* nout;     // outputs in the segment
  const int64_t* segid;    // global (group, segment) index
  const int32_t* abort = nullptr;  // device flag or null: set, the recombination exits at once
  const int32_t* sgroup = nullptr; // group whose sources drive the column (group holds its
                                   // state slot; the two differ only for batched ramps)
};
constexpr int kRampBatch = 256;  // ramp columns per batch when there are more

struct SourceTable {
  const int32_t* grp_ptr;  // [n_groups+1] into grp_src
  const int32_t* grp_src;  // sources grouped by group
  const int32_t* node;     // permuted node of each source
  const int32_t* pwl_off;
  const double* pwl_t;
  const double* pwl_v;
};

// Trapezoidal baseline (k_trap.cu).  b = dc (or 0) + B u(t) over all sources;
// Y[.][0] = c x - g G x + g (bp + bn) with G in CSR; x = Y[.][0] (and output
// row `row` of Xp when row >= 0).  Permuted node order throughout.
void tr_input(double* b, const double* dc, const SourceTable& src, int n_src, double t, int64_t n,
              cudaStream_t st);
void tr_rhs(double* Y, int ldy, const double* x, const int64_t* rowptr, const int32_t* col,
            const double* val, const double* c, double g, const double* bp, const double* bn,
            int64_t n, cudaStream_t st);
void tr_store(double* x, const double* Y, int ldy, double* Xp, int64_t row, int64_t n,
              cudaStream_t st);


// Y[:, q] = B_k (u_k(l0+L) - u_k(l0)) / L, the input slope on the segment (Y zeroed here)
void build_input_rhs(double* Y, int ldy, int K, const RoundCols& rc, const SourceTable& src,
                     int64_t n, cudaStream_t st);
// z_k = x_k for a group's first segment, else z_k += lprev * z'_k
void advance_z(double* Z, const double* Zp, const double* X, int64_t gstride, const RoundCols& rc,
               int K, int64_t n, cudaStream_t st);
// Y[:, q] = B_k u_k(t) for t = 0 per group (initial states)
void build_initial_rhs(double* Y, int ldy, int K, const SourceTable& src, const int32_t* groups,
                       int64_t n, cudaStream_t st);

// Krylov start: v = x - z + w written to V[vslot][0]; partial sums of |v|^2
void krylov_start(double* Vbase, int64_t vstride, const double* X, const double* Z,
                  const double* W, int64_t gstride, const int32_t* groups, const int32_t* vslots,
                  int K, int64_t n, double* partials, int nchunks, cudaStream_t st);

// Partial dot products of basis slot wslot (w) with slots first..first+nb-1
// for each iterating column; partials laid out [K][kMaxB][nchunks].
void basis_dots(const double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter,
                int K, int first, int nb, int wslot, int64_t n, double* partials, int nchunks,
                cudaStream_t st);
// w -= sum_i h[q][i] v_i  (h from coef, [K][kMaxB])
void basis_update(double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter,
                  int K, int nb, int wslot, const double* h, int64_t n, cudaStream_t st);
// V[wslot] *= scale[q]
void basis_scale(double* Vbase, int64_t vstride, const int32_t* groups, const int32_t* iter,
                 int K, int wslot, const double* scale, int64_t n, cudaStream_t st);

constexpr int kChunk = 4096;  // nodes per reduction chunk

// Small dense per-column work (one CTA per column).
struct SmallState {
  double* Ht;        // [ncol][kMaxB][kMaxM] rational Hessenberg (row-major)
  double* beta;      // [ncol]
  int32_t* m;        // [ncol] current / final Krylov dimension (0 = quiescent)
  int32_t* status;   // [ncol] 0 iterating, 1 converged, 2 breakdown, 3 m_max, 4 quiescent
  double* hbuf;      // [ncol][kMaxB] Gram-Schmidt coefficients of the current pass
  double* scale;     // [ncol] 1/norm for normalisation
  int32_t krylov = 0;   // Krylov space: 0 rational, 1 inverted, 2 standard (exponent map)
  double rscale = 1.0;  // factor on h_{m+1,m} in the residual: 1, 1/gamma, gamma
};

// finish the start vector: beta = sqrt(sum partials), scale = 1/beta, status;
// writes the list of non-quiescent columns and its count
void start_finish(const double* partials, int nchunks, int K, SmallState ss, const int32_t* groups,
                  int32_t* iter_out, int32_t* iter_grp, int32_t* iter_count, cudaStream_t st);
// reduce dot partials into hbuf (and accumulate into Ht column j when acc != 0)
void reduce_dots(const double* partials, int nchunks, int K, int nb, const int32_t* iter,
                 SmallState ss, int j, int mode, cudaStream_t st);
// residual test after step j (m = j+1): decides status per column; writes
// the compacted list of still-iterating columns and its count
// Guard of a recorded (graph) run: when *count differs from the count the
// recorded launches were sized for, raise *flag and point the entries
// [*count, expected) of iter / iter_grp at column 0 of the round, so that the
// rest of the replay (whose result is then discarded) stays in range.
void expect_count(const int32_t* count, int expected, int32_t* iter, int32_t* iter_grp,
                  const int32_t* vslot, int32_t* flag, cudaStream_t st);
// w = A v = -C^{-1} G v for the standard Krylov space: column q of the batch
// reads slot `jsrc` of its basis and writes slot `jdst` (G in CSR, permuted).
void krylov_apply_A(double* Vb, int64_t vstride, const int32_t* iter_grp, int K, int jsrc, int jdst,
                    const int64_t* rowptr, const int32_t* col, const double* val, const double* c,
                    int64_t n, cudaStream_t st);
void residual_check(SmallState ss, const RoundCols& rc, int K, int j, double gamma, double tol,
                    int m_max, const int32_t* replay, const int32_t* iter_in, int32_t* iter_out,
                    int32_t* iter_grp, int32_t* iter_count, cudaStream_t st);
// record m and status of the round's columns at their global segment ids
void record_segments(const SmallState& ss, const RoundCols& rc, int K, int32_t* m_rec,
                     int32_t* st_rec, cudaStream_t st);
// coefficient vectors beta e^{h H} e_1 for every output of the segment and
// for the segment end; coef [K][ldo][kCoefLd] (slot kMaxM holds h), yend [K][kMaxM].
// With tail_eps > 0 it also writes each column's tail cut: tcut[2q] = outputs,
// from the segment's first, up to the last one with ||y||_2 > tail_eps/2;
// tcut[2q+1] = 1 when pbound[q] <= tail_eps/2 as well (the -P term is dropped
// past the cut too).  With tail_eps = 0, tcut[2q] = the column's output count.
void output_coefficients(SmallState ss, const RoundCols& rc, int K, double gamma, double dt_out,
                         double* coef, int ldo, double* yend, cudaStream_t st,
                         double tail_eps = 0.0, const double* pbound = nullptr,
                         int32_t* tcut = nullptr);
// pbound[2q] = max_i |z_i - w_i| and pbound[2q+1] = max_i |z'_i| over the
// column's group, so that pbound[2q] + L pbound[2q+1] bounds its -P term
// z + h z' - w for every h in [0, L] (a NaN anywhere makes the bound NaN)
void p_bound(const double* Z, const double* Zp, const double* W, int64_t gstride,
             const RoundCols& rc, int K, int64_t n, double* pbound, cudaStream_t st);
size_t small_shared_bytes();
void set_small_smem_limits();
// batched expm for the public test entry point
void expm_batch(int batch, int m, const double* A, const double* h, double* E, cudaStream_t st);

// Recombination + superposition: Xp[o][i] += sum over columns whose segment
// holds o of (V y_o + z + h z' - w)   (h = t_o - l0).  With tcut (the tail
// cuts of output_coefficients), an output tile that starts at or past a
// column's cut takes the column without V y, or not at all when the column's
// -P term is dropped as well.
void recombine(double* Xp, int64_t n, int n_times, const double* Vbase, int64_t vstride,
               const double* Z, const double* Zp, const double* W, int64_t gstride,
               const RoundCols& rc, const int32_t* mcol, const double* coef, int ldo, int K,
               int obeg_min, int oend_max, double dt_out, cudaStream_t st,
               const int32_t* tcut = nullptr);
// next state x_k = V y_end + z + L z' - w
void next_state(double* X, const double* Vbase, int64_t vstride, const double* Z, const double* Zp,
                const double* W, int64_t gstride, const RoundCols& rc, const int32_t* mcol,
                const double* yend, int K, int64_t n, cudaStream_t st);
// Tensor-core recombination of the V y part (k_recombine_tc.cu): error-free
// 6-bit slices of V (per node) and of the coefficients (per output) in bf16,
// tcgen05 MMAs into FP32 accumulators that stay exact integers, exact
// integer combination, FP64 result added into Xp.  Scratch of a context,
// sized at setup for rounds of up to kdim_cap basis vectors.
constexpr int kTcMaxKdim = 2048;  // basis vectors of one round the scratch may be sized for
constexpr int kTcMinKdim = 16;    // below this the FP64 kernel is cheaper
struct TcScratch {
  void* slices = nullptr;       // V and coefficient slices in the MMA tile layout
  int64_t* kmap = nullptr;      // [kdim_cap] basis vector -> offset in Vbase
  int32_t* kq = nullptr;        // [kdim_cap] basis vector -> (column << 5) | index
  double* rowscale = nullptr;   // [n] power-of-two scale of each node's basis values
  double* colscale = nullptr;   // [output tiles x 48] scale of each output's coefficients
  int32_t* err = nullptr;       // raised when a bounded wait of the MMA kernel gives up
  int kdim_cap = 0;
};
size_t tc_slices_bytes(int64_t n, int kdim, int nouts);
void tc_set_limits();
// Xp[o][i] += sum over the round's columns q and j < mcol[q] of V_q[j][i] y_q(o)[j]
// for o in [obeg_min, oend_max) (the columns' own output ranges); kdim = sum
// of mcol.  Returns the number of kernels launched.
int recombine_tc(double* Xp, int64_t n, const double* Vbase, int64_t vstride, const RoundCols& rc,
                 const int32_t* mcol, const double* coef, int ldo, int K, int kdim, int obeg_min,
                 int oend_max, const TcScratch& ts, cudaStream_t st);

// The -P terms z + h z' - w of a round's columns at their outputs, added into
// Xp by one sweep over the outputs per node; events ev_o / ev_q (nev, sorted
// by output) mark where a column's output range starts (q + 1) or ends (-(q + 1)).
void recombine_p(double* Xp, int64_t n, const double* Z, const double* Zp, const double* W,
                 int64_t gstride, const RoundCols& rc, const int32_t* ev_o, const int32_t* ev_q,
                 int nev, int o_begin, int o_end, double dt_out, cudaStream_t st);
constexpr double kTcMinCover = 0.25;  // least share of a round's (column, output) pairs its
                                      // columns cover for the dense tensor-core product to pay

// Adjoint checkpoints: CK[q] = {X[groups[q]], Z[groups[q]]} ([K][2][n]), or the
// reverse copy when restore is set (X, Z per group, [G][n]).
void checkpoint_states(double* CK, double* X, double* Z, const int32_t* groups, int K, int64_t n,
                       bool restore, cudaStream_t st);
// Xp[o][i] = base[i] for all o
void fill_rows(double* Xp, const double* base, int64_t n, int n_times, cudaStream_t st);
// Xp[0][i] += sum_q Y[i][q]
void add_row_sum(double* Xp, const double* Y, int ldy, int K, int64_t n, cudaStream_t st);
// out[o][r] = Xp[o][map[r]]
void permute_out(double* out, const double* Xp, const int32_t* map, int64_t nrows, int64_t n,
                 int n_times, cudaStream_t st);

// ---------------------------------------------------------------------------
// Adjoint (reverse of the batched forward; see k_adjoint.cu)
// ---------------------------------------------------------------------------
// Per-column work slots: qbar_0..qbar_{kMaxB-1}, then zbar, zbar', wbar, rbar, abar.
constexpr int kWZ = kMaxB, kWZp = kMaxB + 1, kWW = kMaxB + 2, kWR = kMaxB + 3, kWA = kMaxB + 4;
constexpr int kWSlots = kMaxB + 5;

// One reverse round: the columns of a forward round, with the forward tape.
struct AdjRound {
  const int32_t* rec;     // per column: tape record (its basis slot)
  const int32_t* group;
  const int32_t* m;       // per column Krylov dimension
  const int32_t* obeg;
  const int32_t* nout;
  const int32_t* seg;
  const double* l0;
  const double* len;
  const double* hfirst;
  const double* V;        // tape bases [records][kMaxB][n]
  int64_t vstride;
  const double* A;        // tape solve outputs a_k [records][kMaxM][n]
  int64_t astride;
  const double* Zp;       // tape z' [records][n]
  const double* Ht;       // tape Hessenbergs [records][kMaxB][kMaxM]
  const double* beta;     // tape norms [records]
  int64_t n;
  double dt;
};
struct AdjWork {
  double* work;           // [K][kWSlots][n]
  int64_t wstride;
  double* XB;             // [G][n] xbar flowing into the group's previous segment
  double* CARRY;          // [G][n] zbar carried to the previous segment (z_{j+1} = z_j + L_j z'_j)
  double* CB;             // [G][n] capacitance adjoint per group
};
// out[q][i] = a_q . b_q[i] for i < nb, a_q = a + a_idx[q]*a_stride + a_slot*n, likewise b
struct AdjDots {
  const double* a;
  int64_t a_stride;
  const int32_t* a_idx;
  int a_slot;
  const double* b;
  int64_t b_stride;
  const int32_t* b_idx;
  int b_slot;
  const int32_t* cols;    // columns to process (null: 0..K-1)
};

void tape_small(const SmallState& ss, const RoundCols& rc, int K, double* THt, double* Tbeta,
                cudaStream_t st);
size_t adj_small_shared_bytes();
void adj_set_limits();
void adj_obs(const AdjRound& ar, int K, const double* xbar, const int32_t* map, int nrows,
             double* ybo, int ldo, double* S1, double* S2, cudaStream_t st);
void adj_dots(const AdjDots& d, int K, int nb, int64_t n, double* partials, int nchunks, double* out,
              cudaStream_t st);
void adj_small(const AdjRound& ar, int K, double gamma, const double* ybo, int ldo,
               const double* ybL, double* yout, double* yL, double* Htbar, double* betabar,
               cudaStream_t st);
void adj_build(const AdjRound& ar, const AdjWork& aw, int K, const double* yL, const double* xbar,
               const int32_t* map, int nrows, const double* yout, int ldo, const double* S1,
               const double* S2, cudaStream_t st);
void adj_rbar(const AdjRound& ar, const AdjWork& aw, const int32_t* act, int Ka, int k,
              const double* d1, const double* Htbar, cudaStream_t st);
void adj_abar(const AdjRound& ar, const AdjWork& aw, const int32_t* act, int Ka, int k,
              const double* hdot, const double* Htbar, cudaStream_t st);
void adj_after_m(const AdjRound& ar, const AdjWork& aw, const int32_t* act, int Ka, int k,
                 const double* Y, int ldy, const double* c, cudaStream_t st);
void adj_vbar(const AdjRound& ar, const AdjWork& aw, int K, const double* d0, const double* betabar,
              cudaStream_t st);
void adj_after_w(const AdjRound& ar, const AdjWork& aw, int K, const double* Y, int ldy,
                 const double* c, cudaStream_t st);
void adj_sources(const AdjRound& ar, int K, const SourceTable& src, const double* Y, int ldy,
                 double* ampbar, cudaStream_t st);
void adj_init_sources(const int32_t* groups, int K, const SourceTable& src, const double* Y, int ldy,
                      double* ampbar, cudaStream_t st);
void adj_x0_obs(const int32_t* groups, int K, double* XB, int64_t n, const double* xbar0,
                const int32_t* map, int nrows, cudaStream_t st);
void adj_csum(const double* CB, int G, int64_t n, const int32_t* perm, double* dc, cudaStream_t st);

// Resident rounds (k_resident.cu): on small grids one CTA runs a column's
// whole segment, its triangular substitutions level by level inside the CTA.
// The path keeps its own copy of each factor's panels stored level by level
// (leaves first), D^{-1} folded into the diagonal blocks' forward rows, and a
// plan small enough to sit in the CTA's shared memory for the whole kernel
// (every global load then goes to panel entries; a load from L2 costs a CTA
// with one column far more than the arithmetic):
//   sups[s]: the supernode's panel offset p in the copies, first node f,
//     width w, rows ld, its first forward row (rb) and backward column (cb)
//     within its level, and the global number gb of its first row below the
//     diagonal block;
//   fsup / bsup: per level, the supernode of each forward row / backward
//     column (row i = t - rb, column k = t - cb);
//   forward: a diagonal row stores y, a row below the diagonal block stores
//     its product in scratch slot gb + i - w - offs[LB][l]; then target
//     tgt[j] subtracts, in order, the slots tslot[tpp[j-1] .. tpp[j]) (from 0
//     for the level's first target): all products in parallel, each sum in a
//     fixed order (no atomics, reproducible);
//   brows[gb + i - w]: the ancestor node of row i >= w (backward gathers).
// offs[X][l] for X = R, T, C: level l's first forward row, target, backward
// column; FL, BL: lanes per dot product (1, 2, 4 or 8, more on levels with
// few rows); LB: the level's first row below a diagonal block.
constexpr int64_t kResidentMaxN = 8192;
constexpr int kResidentMaxLevels = 64;
constexpr int kResidentThreads = 512;
constexpr int kResOffR = 0, kResOffT = 1, kResOffC = 2, kResOffFL = 3, kResOffBL = 4,
              kResOffLB = 5, kResOffN = 6;
struct ResSup {
  int32_t p, f, w, ld, rb, cb, gb;
};
struct ResFactor {  // one factor's panels in the resident order
  const double* fpan = nullptr;  // column-major per supernode, D^{-1} in the diagonal rows
  const double* bpan = nullptr;  // row-major per supernode
};
// The plan is one blob (copied to shared memory at kernel start); o_* are
// byte offsets of its sections, each 16-byte aligned.
struct ResidentPlan {
  const unsigned char* blob = nullptr;
  int32_t bytes = 0;
  int32_t o_offs = 0, o_sups = 0, o_fsup = 0, o_bsup = 0, o_tgt = 0, o_tpp = 0, o_tslot = 0,
          o_brows = 0;
  int32_t nlev = 0;
  int32_t uslots = 0;  // largest number of below-diagonal rows of a level
};
// where one supernode's panel goes in the resident copies
struct ResStoreSup {
  int64_t src, fdst, bdst;
  int32_t f, w, ld;
};
struct ResidentArgs {
  ResFactor F1;          // X1 of the Krylov space (C + gamma G, or G for the inverted space)
  ResFactor FG;          // G
  ResidentPlan plan;
  double* Vb;            // basis slots, vstride apart
  int64_t vstride;
  double *X, *Z, *Zp, *W;  // per state slot, n apart
  const double* cperm;   // capacitances in the factor's order
  SourceTable src;
  RoundCols rc;
  SmallState ss;
  double* coef;
  int32_t ldo;
  double* yend;
  int32_t *m_rec, *st_rec;
  const int32_t* replay;
  double gamma, tol, dt_out;
  int32_t m_max;
  int64_t n;
  // z' and w of column q at zpre + q n, wpre + q n: written by
  // resident_inputs, read by resident_round (null: the round solves them)
  double* zpre = nullptr;
  double* wpre = nullptr;
};
// the resident copies of factor F (fpan, bpan: as many doubles as F's
// panels) from the per-supernode map sup[nsup]
void resident_store(const DevFactor& F, const ResStoreSup* sup, int nsup, double* fpan, double* bpan,
                    cudaStream_t st);
// whether a grid of n nodes with plan P fits one CTA's shared memory on this
// device
bool resident_fits(int64_t n, const ResidentPlan& P);
// raise the kernels' shared-memory limits for them (false on failure)
bool resident_set_limits(int64_t n, const ResidentPlan& P);
// one round: K CTAs, column q of rc by CTA q
void resident_round(const ResidentArgs& a, int K, cudaStream_t st);
// the input solves of K columns of rc ahead of their rounds (they depend on
// the sources only): z', w of column q into a.zpre, a.wpre + q n
void resident_inputs(const ResidentArgs& a, int K, cudaStream_t st);
// x_q = F^{-1} b_q for ncols columns, one CTA each: entry i of column q at
// q * ldq + r(i) * ldi with r = perm (new -> old: the caller's order) or the
// identity (the factor's order); b and x may alias
void resident_solve(const ResFactor& F, const ResidentPlan& P, const double* b, double* x,
                    int64_t n, int ncols, int64_t ldi, int64_t ldq, const int32_t* perm,
                    cudaStream_t st);
// best of reps (ms) of one CTA's solve pair x = F^{-1} b (b, x: n doubles of
// the device); -1 on a CUDA error
float resident_time_solve(const ResFactor& F, const ResidentPlan& P, const double* b, double* x,
                          int64_t n, cudaStream_t st, int reps);

// Single-right-hand-side level solves (k_sptrsv_k1.cu).  Per direction, the
// supernodes of every level in launch order (sorted by group size, then
// size) as records, and per level the warps' work: warp j of level l starts
// at row (forward) or column (backward) i0 of record k0 and covers nslot
// consecutive rows of the following records of the same group size, each by
// 2^lg lanes.  fw_off / bw_off (host memory, nlev + 1 each) delimit the
// levels' warps.
struct K1Sup {
  int64_t po, rp;  // panel offset, first entry of the row list
  int32_t f, w, ld, pad;
};
struct K1Warp {
  int32_t k0, i0;
  int16_t lg, nslot;
  int32_t pad;
};
struct K1Plan {
  int32_t nlev = 0, nsup = 0;
  const K1Sup* fsups = nullptr;
  const K1Sup* bsups = nullptr;
  const K1Warp* fwarps = nullptr;
  const K1Warp* bwarps = nullptr;
  const int32_t* fw_off = nullptr;
  const int32_t* bw_off = nullptr;
};
// one solve pair x = F^{-1} b for the single column 0 of Y (node-major, ldy
// apart; Y2 scratch of the same shape): one launch per level and direction,
// chained by programmatic dependent launch; returns the launches
int solve_k1(const DevFactor& F, const K1Plan& P, double* Y, double* Y2, int ldy, cudaStream_t st);

// Wide supernodes of the level solves on the tensor cores (k_sptrsv_tc.cu).
// Per wide supernode: its panel (offset pan, first node f, width w, rows ld,
// row list rp), the row tiles of the forward (ld rows) and backward (w rows)
// products, and the offsets of its panel slices (a_f, a_b: bytes into the
// direction's slice store of the factor) and of its row scales (rs_f, rs_b,
// in doubles).
struct TsSup {
  int64_t pan, rp;
  int32_t f, w, ld, mt_f, mt_b, pad;
  int64_t a_f, a_b, rs_f, rs_b;
};
// One tree level's wide supernodes (indices into the TsSup table) and the
// tiles of its two products: {supernode, row tile | K slice << 16}.
struct TsLevel {
  int32_t nsup = 0, ntile_f = 0, ntile_b = 0;
  const int32_t* list = nullptr;
  const int2* tiles_f = nullptr;
  const int2* tiles_b = nullptr;
};
constexpr int kTsMinWidth = 64;  // default: supernodes at least this wide use the tensor cores
size_t ts_a_bytes(int rows, int kdim);   // panel slices of one product
int ts_row_tiles(int rows);
int ts_k_slices(int kdim);               // CTAs sharing one row tile (split reduction)
void ts_set_limits();
// panel slices and row scales of nsup wide supernodes (max_mt: most row tiles)
void ts_split_panels(const DevFactor& F, const TsSup* sups, int nsup, int max_mt, bool fwd,
                     __nv_bfloat16* A, double* rowscale, cudaStream_t st);
// the wide supernodes of one level, one direction, ncols right-hand sides of
// the solve buffers (Y node-major, Y2 the forward intermediate)
void ts_solve_level(const DevFactor& F, const TsSup* sups, const TsLevel& L, bool fwd,
                    const __nv_bfloat16* A, const double* rowscale, double* Y, double* Y2, int ldy,
                    int ncols, int32_t* err, cudaStream_t st);
// one level launch of the FP64 solve (k_sptrsv.cu), the level's own tuned
// column block
void solve_level(bool fwd, const DevFactor& F, const LevelPlan& L, double* Y, double* Y2, int ldy,
                 int ncols, cudaStream_t st, const SplitScratch* split);

}  // namespace matex
