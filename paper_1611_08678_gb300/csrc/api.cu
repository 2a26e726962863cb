// C ABI (include/abm.h): plans, argument checks, host-side scheduling and the
// launch sequences of the single and batched paths.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda.h>

#include "batched.cuh"
#include "common.cuh"
#include "single.cuh"
#include "status_text.h"

namespace abm {
// kernels (weights.cu, single.cu, batched.cu)
cudaError_t launch_weights(double alpha, int M, double* b, double* a, double* c, double* g,
                           cudaStream_t st);
cudaError_t launch_weights_f32(int M, const double* b, const double* a, float* b32, float* a32,
                               cudaStream_t st);

cudaError_t launch_batched_setup(int sys, const BatchArgs& A, int n_tiles, cudaStream_t st);
cudaError_t launch_batched_near(int sys, const BatchArgs& A, int n_active, long long s, int nb, int qw,
                                int split, cudaStream_t st);
cudaError_t launch_batched_far(int d, abm_precision prec, const BatchArgs& A, int n_active, long long s,
                               cudaStream_t st);
cudaError_t launch_far_tc(int kind, const FarTcArgs& A, int n_active, cudaStream_t st);
cudaError_t launch_build_wx(const double* b, const double* a, long long Mw, long long Lbase, long long Lx,
                            __nv_bfloat16* Wx, cudaStream_t st);
bool make_tmap_bf16(CUtensorMap* out, void* base, unsigned long long inner, unsigned long long rows,
                    unsigned box_rows);
cudaError_t launch_fill_fsh(const double* F, long long s, __nv_bfloat16* Fsh, long long plane, cudaStream_t st);
cudaError_t launch_sum_partials(const double* far, int ksplit, int n_tiles, double* P, double* C, cudaStream_t st);
cudaError_t launch_adjoint_setup(int sys, const AdjArgs& A, int n_tiles, cudaStream_t st);
cudaError_t launch_import_history(int d, const BatchArgs& A, int n_tiles, long long s0, const double* Fin,
                                  long long ldF, long long fin_elems, cudaStream_t st);
cudaError_t launch_export_history(int d, const BatchArgs& A, int n_tiles, long long rows, double* Fout, long long ldF,
                                  long long fout_elems, cudaStream_t st);
cudaError_t launch_adjoint_near(int sys, const AdjArgs& A, int n_active, long long s, int nb, int wpc,
                                int split, cudaStream_t st);
cudaError_t launch_adjoint_finish(int sys, const AdjArgs& A, int M, cudaStream_t st);
}  // namespace abm

using namespace abm;

namespace {

constexpr int kDefaultB = 64;
constexpr int kEventRing = 4;
constexpr int kMaxWeightSets = 24;

struct WeightSet {
  double alpha = 0.0;
  double *b = nullptr, *a = nullptr, *c = nullptr, *g = nullptr;
  float *b32 = nullptr, *a32 = nullptr;
  __nv_bfloat16* Wx = nullptr;  // pre-expanded Toeplitz pieces (tensor-core paths)
  unsigned long long last_use = 0;
};

}  // namespace

struct abm_plan_s {
  abm_system sys;
  int d = 0, np = 0;
  abm_plan_opts o{};
  int B = kDefaultB;
  int device = 0, sms = 0;
  int Mw = 0;                       // weights are generated for lags 0..Mw
  std::vector<WeightSet> wsets;
  unsigned long long use_clock = 0;
  // single trajectory
  double* F1 = nullptr;             // (n_max + B + 1) x d
  int last_single_rows = 0;         // N + 1 of the last single-trajectory solve (abm_history)
  double* far1 = nullptr;           // [2][B][2d]
  double* part1 = nullptr;          // [2][G][B][2d]
  unsigned int* tickets = nullptr;  // [2]
  double* hhat1 = nullptr;          // 1
  int G = 0;                        // CTAs of the stand-alone far kernel
  int Gp = 0;                       // CTAs of the persistent single-trajectory kernel
  double* ppartial = nullptr;       // [kPersistRing][Gp-1][kPersistB][2d]
  unsigned long long* pflags = nullptr;  // [1 + kPersistRing]
  cudaStream_t side = nullptr;
  cudaEvent_t ev_near[kEventRing] = {}, ev_far[kEventRing] = {}, ev_start = nullptr;
  // batched
  int max_tiles = 0;
  double* Fb = nullptr;
  float* Fb32 = nullptr;
  size_t fb_cap = 0;                // elements
  double* farb = nullptr;
  size_t farb_cap = 0;
  unsigned int* far_ticket = nullptr;  // per column tile (2 per tile for the adjoint), zero between launches
  TileDesc* d_tiles = nullptr;
  double* d_h = nullptr;
  int* d_N = nullptr;
  double* d_hhat = nullptr;         // [max_batch][kMaxD]
  // per order group and component, entry [group * kMaxD + component]
  double* d_balpha = nullptr;
  double* d_bg = nullptr;           // gathered g
  int* d_btaylor = nullptr;         // per group: bit c = component c has order above one
  const double** d_bptr = nullptr;  // [3][kMaxWeightSets * kMaxD] b, a, c pointers
  const float** d_b32ptr = nullptr; // [2][kMaxWeightSets * kMaxD]
  // tensor-core far history (BF16 split precisions)
  __nv_bfloat16* Fsh = nullptr;     // [3][max_tiles*96][fsh_ld]
  long long fsh_ld = 0;
  long long Lbase = 0, Lx = 0;      // pre-expanded Toeplitz geometry
  CUtensorMap* d_tmapW = nullptr;   // [kMaxWeightSets][3]
  CUtensorMap* d_tmapF = nullptr;   // [3]
  // adjoint workspace (allocated by the first abm_adjoint call)
  double* Xadj = nullptr;           // FP64 mu~ / lambda~ histories, 2 tiles per forward tile
  __nv_bfloat16* Xsh = nullptr;     // their BF16 split planes (tensor-core paths)
  CUtensorMap* d_tmapX = nullptr;   // [3]
  TileDesc* d_atiles = nullptr;     // [2 * max_tiles]
  double *acc_dp = nullptr, *acc_dy0 = nullptr, *phi0c = nullptr;
  // host-buffer batched solve (abm_solve_batched_host; allocated by its first call)
  double *hio_params = nullptr, *hio_y0 = nullptr, *hio_Y = nullptr, *hio_YP = nullptr;
  double *hio_Y1 = nullptr, *hio_YP1 = nullptr;  // abm_solve_host (single trajectory)
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> hio_ev;  // per time tile in which trajectories finish
  cudaEvent_t hio_done = nullptr;
  // CUDA graph of the batched launch sequence (opts.use_graph)
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  bool capturing = false;
  unsigned long long* status = nullptr;
  std::string err;
  // tracing: launches per kernel kind, optional event pairs around each launch
  long long launches[ABM_KERNEL_KINDS] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<std::pair<int, size_t>> ev_used;  // (kind, pool index)
};

namespace {

abm_status fail(abm_plan p, abm_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

abm_status cuda_fail(abm_plan p, cudaError_t e, const char* what) {
  return fail(p, e == cudaErrorMemoryAllocation ? ABM_ERR_OOM : ABM_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, what); \
  } while (0)

int sys_dim(abm_system s) {
  switch (s) {
    case ABM_SYS_LINEAR: case ABM_SYS_MANUFACTURED: return 1;
    case ABM_SYS_LORENZ: case ABM_SYS_CHEN: case ABM_SYS_ROSSLER: case ABM_SYS_FINANCIAL: return 3;
    case ABM_SYS_HINDMARSH_ROSE: return 3;
  }
  return -1;
}

int sys_nparams(abm_system s) {
  switch (s) {
    case ABM_SYS_LINEAR: return 3;
    case ABM_SYS_MANUFACTURED: return 9;
    case ABM_SYS_LORENZ: case ABM_SYS_CHEN: case ABM_SYS_ROSSLER: case ABM_SYS_FINANCIAL: return 3;
    case ABM_SYS_HINDMARSH_ROSE: return 8;
  }
  return -1;
}

bool alpha_ok(double a) { return std::isfinite(a) && a > 0.0 && a <= 1.0; }
// orders of the general problem (abm_solve_ext, abm_solve_batched_ext)
bool order_ok(double a) { return std::isfinite(a) && a > 0.0 && a <= 2.0; }

// Tracing: opens an event pair before a launch of `kind` (when profiling) and
// closes it after; counts the launch.
struct Trace {
  abm_plan p;
  int kind;
  cudaStream_t st;
  size_t idx = (size_t)-1;
  Trace(abm_plan p_, int kind_, cudaStream_t st_) : p(p_), kind(kind_), st(st_) {
    p->launches[kind] += 1;
    if (!p->o.profile || p->capturing) return;
    if (p->ev_used.size() >= p->ev_pool.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      p->ev_pool.push_back({a, b});
    }
    idx = p->ev_used.size();
    p->ev_used.push_back({kind, idx});
    cudaEventRecord(p->ev_pool[idx].first, st);
  }
  ~Trace() {
    if (idx != (size_t)-1) cudaEventRecord(p->ev_pool[idx].second, st);
  }
};

// Weight vectors for one alpha (cached; least recently used set is reused).
abm_status get_weights(abm_plan p, double alpha, cudaStream_t st, WeightSet** out) {
  for (auto& w : p->wsets)
    if (w.b && w.alpha == alpha) { w.last_use = ++p->use_clock; *out = &w; return ABM_OK; }
  WeightSet* slot = nullptr;
  for (auto& w : p->wsets)
    if (!w.b) { slot = &w; break; }
  if (!slot) {
    slot = &p->wsets[0];
    for (auto& w : p->wsets)
      if (w.last_use < slot->last_use) slot = &w;
  }
  if (!slot->b) {
    size_t n = (size_t)p->Mw + 1;
    CK(cudaMalloc(&slot->b, n * sizeof(double)), "weights");
    CK(cudaMalloc(&slot->a, n * sizeof(double)), "weights");
    CK(cudaMalloc(&slot->c, n * sizeof(double)), "weights");
    CK(cudaMalloc(&slot->g, sizeof(double)), "weights");
    CK(cudaMalloc(&slot->b32, n * sizeof(float)), "weights");
    CK(cudaMalloc(&slot->a32, n * sizeof(float)), "weights");
  }
  slot->alpha = alpha;
  slot->last_use = ++p->use_clock;
  if (p->Fsh && !slot->Wx)
    CK(cudaMalloc(&slot->Wx, (size_t)3 * 128 * p->Lx * sizeof(__nv_bfloat16)), "toeplitz pieces");
  {
    Trace tr(p, ABM_KERNEL_WEIGHTS, st);
    CK(launch_weights(alpha, p->Mw, slot->b, slot->a, slot->c, slot->g, st), "weights kernel");
    CK(launch_weights_f32(p->Mw, slot->b, slot->a, slot->b32, slot->a32, st), "weights f32");
    if (p->Fsh) CK(launch_build_wx(slot->b, slot->a, p->Mw, p->Lbase, p->Lx, slot->Wx, st), "toeplitz pieces kernel");
  }
  *out = slot;
  return ABM_OK;
}


// History split of the tensor-core far kernel (CTAs per column tile).  The
// kernel runs one CTA per SM, so n_tiles * ks CTAs take ceil(n_tiles * ks /
// sms) waves, each as long as one CTA: a fixed part (TMEM and barrier setup,
// pipeline fill, the FP64 reductions at the end; about kFarCtaSetupBlocks
// K blocks of streaming) plus its ceil(nkb / ks) K blocks.  Picks the split
// with the least modelled time among those within max_waves times the waves
// of the unsplit launch: a split that fills a partial last wave (512 tiles
// on 152 SMs: 3.4 waves unsplit, 6.7 split in two) is allowed, one that only
// multiplies short CTAs is not.
constexpr double kFarCtaSetupBlocks = 6.0;
int far_ksplit(int n_tiles, int nkb, int sms, int max_waves) {
  int best = 1;
  double best_cost = 1e300;
  const long long cap = (long long)max_waves * (((long long)n_tiles + sms - 1) / sms);
  for (int ks = 1; ks <= nkb; ++ks) {
    const long long waves = ((long long)n_tiles * ks + sms - 1) / sms;
    if (ks > 1 && waves > cap) break;
    const double cost = (double)waves * (kFarCtaSetupBlocks + (double)((nkb + ks - 1) / ks));
    if (cost < best_cost) {
      best_cost = cost;
      best = ks;
    }
  }
  return best;
}

// Tensor-core far kernel of the plan's precision: 3 = BF16x3, 6 = BF16x6.
int far_kind(const abm_plan p) { return p->o.prec == ABM_PREC_BF16X3_FAR ? 3 : 6; }

FarTcArgs far_tc_args(abm_plan p, const TileDesc* tiles, const CUtensorMap* tmapF, long long s, int n_tiles, int ks) {
  FarTcArgs T{};
  T.tiles = tiles;
  T.tmapW = p->d_tmapW;
  T.tmapF = tmapF;
  T.far = p->farb;
  T.status = p->status;
  T.s = s;
  T.Lbase = p->Lbase;
  T.budget = p->o.spin_timeout_cycles > 0 ? p->o.spin_timeout_cycles : 4000000000LL;
  T.n_tiles = n_tiles;
  T.ksplit = ks;
  T.f_kblocks = (int)(p->fsh_ld / 64);
  const long long gcols = (long long)p->max_tiles * kTrajPerTile * p->d;
  T.f_map_rows = gcols * (p->fsh_ld / 64) * (tmapF == p->d_tmapX ? 2 : 1);  // adjoint planes: 2 tiles per tile
  T.w_map_rows = 2 * p->Lx;
  T.far_elems = (long long)p->farb_cap;
  return T;
}

// abm_far_history on a tensor-core plan: one column tile of 96 columns, history
// rows [1, s) with s a multiple of 64 (the tensor path always covers whole
// 64-row blocks from row 0, whose BF16 copy is zero).
abm_status far_history_tc(abm_plan p, double alpha, const double* F, long long rows, long long cols, long long s,
                          int B, long long k_lo, long long k_hi, double* P, double* C, cudaStream_t st) {
  if (cols != 96 || B != 64 || k_lo != 1 || k_hi != s || s % 64 != 0 || s < 64 || s > p->Lbase || rows < s ||
      p->max_tiles < 1)
    return fail(p, ABM_ERR_INVALID_ARG,
                "abm_far_history (tensor-core plan): needs cols = 96, B = 64, k_lo = 1, k_hi = s, s a multiple of 64");
  WeightSet* w;
  abm_status rs = get_weights(p, alpha, st, &w);
  if (rs) return rs;
  const long long gcols = (long long)p->max_tiles * kTrajPerTile * p->d;
  CK(launch_fill_fsh(F, s, p->Fsh, gcols * p->fsh_ld, st), "fill history pieces");
  CUtensorMap mw[3];
  for (int q = 0; q < 3; ++q)
    if (!make_tmap_bf16(&mw[q], w->Wx + (size_t)q * 128 * p->Lx, 64, (unsigned long long)(2 * p->Lx), 128))
      return fail(p, ABM_ERR_CUDA, "abm_far_history: tensor map");
  CK(cudaMemcpyAsync(p->d_tmapW, mw, sizeof(mw), cudaMemcpyHostToDevice, st), "tmaps");
  TileDesc td{};
  for (int l = 0; l < kTrajPerTile; ++l) td.traj[l] = l;
  td.bucket = 0;
  td.slot = 0;
  td.n_tile = (int)s + 64;
  CK(cudaMemcpyAsync(p->d_tiles, &td, sizeof(td), cudaMemcpyHostToDevice, st), "tile");
  const int nkb_total = (int)(s / 64);
  const int ks = far_ksplit(1, nkb_total, p->sms, 2);
  CK(cudaMemsetAsync(p->farb, 0, (size_t)2 * 64 * 96 * sizeof(double), st), "far sums reset");
  FarTcArgs T = far_tc_args(p, p->d_tiles, p->d_tmapF, s, 1, ks);
  CK(launch_far_tc(far_kind(p), T, 1, st), "tensor-core far kernel");
  CK(launch_sum_partials(p->farb, ks, 1, P, C, st), "partial sums");
  CK(cudaStreamSynchronize(st), "synchronize");  // the host-staged tile descriptor must outlive the copy
  return ABM_OK;
}

// Host-side scheduling shared by the batched solve and its adjoint: argument
// checks, order groups (trajectories with the same order per component; one
// weight set per distinct order), column tiles of 32 trajectories ordered by
// N, history offsets, and the device tables the kernels read.
struct Sched {
  std::vector<std::array<double, kMaxD>> groups;  // orders per group and component
  std::vector<WeightSet*> ws;                     // [group * kMaxD + component]
  std::vector<TileDesc> tiles;
  int n_tiles = 0, nmax = 0, ksplit = 1;
  bool per_comp = false;                          // some group's orders differ per component
  size_t hist_elems = 0;
  int M = 0;
};

// alpha: M orders (astride = 1, every component) or M x d (astride = d), each
// in (0, amax].
abm_status schedule_batch(abm_plan p, int M, const double* alpha, int astride, double amax, const double* h,
                          const int* N, long long ldY, cudaStream_t st, Sched& S, const char* who) {
  const int B = p->B, d = p->d;
  auto order = [&](int i, int c) { return alpha[(size_t)i * astride + (astride > 1 ? c : 0)]; };
  int& nmax = S.nmax;
  nmax = 0;
  for (int i = 0; i < M; ++i) {
    bool ok = std::isfinite(h[i]) && h[i] > 0.0 && N[i] >= 1 && N[i] <= p->o.n_max;
    for (int c = 0; c < d; ++c) ok = ok && std::isfinite(order(i, c)) && order(i, c) > 0.0 && order(i, c) <= amax;
    if (!ok)
      return fail(p, ABM_ERR_INVALID_ARG, std::string(who) + ": trajectory " + std::to_string(i) + " needs orders in (0," +
                                              (amax > 1.0 ? "2" : "1") + "], finite h > 0, 1 <= N <= n_max");
    nmax = std::max(nmax, N[i]);
  }
  if (ldY < (long long)nmax + 1) return fail(p, ABM_ERR_INVALID_ARG, std::string(who) + ": ldY < max(N)+1");
  // ---- order groups ----
  std::vector<int> group_of(M);
  std::vector<double> values;  // distinct orders (one weight set each)
  for (int i = 0; i < M; ++i) {
    std::array<double, kMaxD> t{};
    for (int c = 0; c < kMaxD; ++c) t[c] = order(i, c < d ? c : 0);
    size_t g = std::find(S.groups.begin(), S.groups.end(), t) - S.groups.begin();
    if (g == S.groups.size()) S.groups.push_back(t);
    group_of[i] = (int)g;
    for (int c = 0; c < d; ++c)
      if (std::find(values.begin(), values.end(), t[c]) == values.end()) values.push_back(t[c]);
  }
  S.M = M;
  const int n_groups = (int)S.groups.size();
  if (n_groups > kMaxWeightSets || (int)values.size() > kMaxWeightSets)
    return fail(p, ABM_ERR_UNSUPPORTED, std::string(who) + ": more than " + std::to_string(kMaxWeightSets) +
                                            " distinct orders or order groups");
  for (const auto& t : S.groups)
    for (int c = 1; c < d; ++c)
      if (t[c] != t[0]) S.per_comp = true;
  if (S.per_comp && p->Fsh)
    return fail(p, ABM_ERR_UNSUPPORTED, std::string(who) + ": the tensor-core far history (BF16X3/X6) takes one order "
                                            "per trajectory; orders that differ per component need an FP64 or FP32 plan");
  std::vector<WeightSet*>& ws = S.ws;
  ws.assign((size_t)n_groups * kMaxD, nullptr);
  for (int g = 0; g < n_groups; ++g)
    for (int c = 0; c < d; ++c) {
      // distinct orders <= the number of weight slots, so the least recently
      // used slot get_weights reuses never holds an order of this batch
      abm_status rs = get_weights(p, S.groups[g][c], st, &ws[(size_t)g * kMaxD + c]);
      if (rs) return rs;
    }
  for (int g = 0; g < n_groups; ++g)
    for (int c = d; c < kMaxD; ++c) ws[(size_t)g * kMaxD + c] = ws[(size_t)g * kMaxD];
  // ---- column tiles: per group, ordered by N descending, 32 trajectories each ----
  std::vector<TileDesc>& tiles = S.tiles;
  tiles.clear();
  for (int g = 0; g < n_groups; ++g) {
    std::vector<int> idx;
    for (int i = 0; i < M; ++i)
      if (group_of[i] == g) idx.push_back(i);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return N[x] > N[y]; });
    for (size_t q = 0; q < idx.size(); q += kTrajPerTile) {
      TileDesc t{};
      for (int l = 0; l < kTrajPerTile; ++l) t.traj[l] = (q + l < idx.size()) ? idx[q + l] : -1;
      t.bucket = g;
      t.n_tile = N[idx[q]];
      tiles.push_back(t);
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const TileDesc& x, const TileDesc& y) { return x.n_tile > y.n_tile; });
  for (size_t t = 0; t < tiles.size(); ++t) tiles[t].slot = (int)t;
  if ((int)tiles.size() > p->max_tiles)
    return fail(p, ABM_ERR_UNSUPPORTED, std::string(who) + ": too many column tiles for this plan");
  size_t off = 0;
  for (auto& t : tiles) {
    t.f_off = (long long)off;
    long long rows = (long long)((t.n_tile + B - 1) / B) * B + 1;
    off += (size_t)rows * kTrajPerTile * d;
  }
  if (off > p->fb_cap) return fail(p, ABM_ERR_UNSUPPORTED, std::string(who) + ": history exceeds workspace");
  const int n_tiles = (int)tiles.size();
  S.n_tiles = n_tiles;
  S.hist_elems = off;
  int& ksplit = S.ksplit;
  ksplit = std::max(1, std::min(16, (2 * p->sms + n_tiles - 1) / n_tiles));
  while ((size_t)ksplit * n_tiles * 2 * B * kTrajPerTile * d > p->farb_cap && ksplit > 1) --ksplit;
  // ---- device tables: entry [group * kMaxD + component] ----
  const size_t NT = (size_t)kMaxWeightSets * kMaxD;
  std::vector<double> balpha(NT, 0.0);
  std::vector<int> btaylor(kMaxWeightSets, 0);
  std::vector<const double*> bptr(3 * NT, nullptr);
  std::vector<const float*> b32ptr(2 * NT, nullptr);
  for (int g = 0; g < n_groups; ++g)
    for (int c = 0; c < kMaxD; ++c) {
      const size_t e = (size_t)g * kMaxD + c;
      const WeightSet* w = ws[e];
      balpha[e] = S.groups[g][c];
      if (c < d && S.groups[g][c] > 1.0) btaylor[g] |= 1 << c;
      bptr[e] = w->b;
      bptr[NT + e] = w->a;
      bptr[2 * NT + e] = w->c;
      b32ptr[e] = w->b32;
      b32ptr[NT + e] = w->a32;
      CK(cudaMemcpyAsync(p->d_bg + e, w->g, sizeof(double), cudaMemcpyDeviceToDevice, st), "g copy");
    }
  CK(cudaMemcpyAsync(p->d_tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, st), "tiles");
  CK(cudaMemcpyAsync(p->d_h, h, M * sizeof(double), cudaMemcpyHostToDevice, st), "h");
  CK(cudaMemcpyAsync(p->d_N, N, M * sizeof(int), cudaMemcpyHostToDevice, st), "N");
  CK(cudaMemcpyAsync(p->d_balpha, balpha.data(), n_groups * kMaxD * sizeof(double), cudaMemcpyHostToDevice, st),
     "alpha");
  CK(cudaMemcpyAsync(p->d_btaylor, btaylor.data(), n_groups * sizeof(int), cudaMemcpyHostToDevice, st), "taylor");
  CK(cudaMemcpyAsync(p->d_bptr, bptr.data(), bptr.size() * sizeof(double*), cudaMemcpyHostToDevice, st), "ptrs");
  CK(cudaMemcpyAsync(p->d_b32ptr, b32ptr.data(), b32ptr.size() * sizeof(float*), cudaMemcpyHostToDevice, st), "ptrs");
  if (p->Fsh) {
    std::vector<CUtensorMap> mw((size_t)n_groups * 3);
    for (int g = 0; g < n_groups; ++g)
      for (int q = 0; q < 3; ++q)
        if (!make_tmap_bf16(&mw[g * 3 + q], ws[(size_t)g * kMaxD]->Wx + (size_t)q * 128 * p->Lx, 64,
                            (unsigned long long)(2 * p->Lx), 128))
          return fail(p, ABM_ERR_CUDA, std::string(who) + ": tensor map of the Toeplitz pieces");
    CK(cudaMemcpyAsync(p->d_tmapW, mw.data(), mw.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st), "tmaps");
  }
  return ABM_OK;
}

// Copy-out of finished rows to host memory while later time tiles run
// (abm_solve_batched_host).  ops[j] lists the copies issued behind time tile
// j: rows lo..hi of the trajectories i0 .. i0+n-1 (one 2D copy: n rows of the
// trajectory dimension, each (hi - lo + 1) * d doubles).
struct CopyOp {
  int i0, n;
  long long lo, hi;
};
struct HostCopyOut {
  std::vector<std::vector<CopyOp>> ops;
  double *Yh = nullptr, *YPh = nullptr;  // host, leading dimension ldh
  long long ldh = 0;
  const double *Yd = nullptr, *YPd = nullptr;  // device, leading dimension ldd
  long long ldd = 0;
};

// The copy plan: after time tile j (rows up to e = (j+1) B are final), a
// trajectory that ends in the tile copies its remaining rows up to N_i, and
// the still-running trajectories copy their rows up to e when they form at
// most kMaxRuns runs of consecutive indices (uniform N: one 2D copy per tile,
// so almost all of the output crosses the host link while the solve runs;
// scattered N: they wait for their own last tile).  Runs of consecutive
// indices with equal row ranges share one 2D copy.
constexpr int kMaxRuns = 32;
std::vector<std::vector<CopyOp>> plan_copy_out(int M, const int* N, int B, int ntime) {
  std::vector<std::vector<CopyOp>> ops(ntime);
  std::vector<long long> copied(M, -1);  // last row already copied
  auto emit = [&](int j, const std::vector<std::pair<int, long long>>& todo) {  // (trajectory, last row)
    for (size_t k = 0; k < todo.size();) {
      const int i0 = todo[k].first;
      const long long lo = copied[i0] + 1, hi = todo[k].second;
      size_t m = k + 1;
      while (m < todo.size() && todo[m].first == todo[m - 1].first + 1 && todo[m].second == hi &&
             copied[todo[m].first] + 1 == lo)
        ++m;
      ops[j].push_back({i0, (int)(m - k), lo, hi});
      for (size_t q = k; q < m; ++q) copied[todo[q].first] = hi;
      k = m;
    }
  };
  for (int j = 0; j < ntime; ++j) {
    const long long s = (long long)j * B, e = s + B;
    std::vector<std::pair<int, long long>> ending, running;
    int runs = 0;
    for (int i = 0; i < M; ++i) {
      if (N[i] <= s) continue;
      if (N[i] <= e) {
        ending.push_back({i, N[i]});
      } else {
        if (running.empty() || running.back().first != i - 1) ++runs;
        running.push_back({i, e});
      }
    }
    emit(j, ending);
    if (runs <= kMaxRuns) emit(j, running);
  }
  return ops;
}

// The far / near launch sequence of one batched solve on stream st (tables
// already on the device); with out, each time tile's finished trajectories
// are copied to the host on the plan's copy stream behind that tile.
abm_status enqueue_batched(abm_plan p, const Sched& S, BatchArgs A, cudaStream_t st,
                           const HostCopyOut* out = nullptr) {
  const int B = p->B, d = p->d;
  const bool tc_prec = p->Fsh != nullptr;
  const std::vector<TileDesc>& tiles = S.tiles;
  CK(launch_batched_setup(p->sys, A, S.n_tiles, st), "setup kernel");
  const int ntime = (S.nmax + B - 1) / B;
  int n_active = S.n_tiles;
  const int j0 = (int)(A.resume_row / B);  // resume: rows 0..j0 B come from the imported history
  for (int j = j0; j < ntime; ++j) {
    const long long s = (long long)j * B;
    while (n_active > 0 && tiles[n_active - 1].n_tile <= s) --n_active;
    if (n_active == 0) break;
    A.n_tiles = n_active;  // far sums of this time tile: [ksplit][n_active][2][B][cols]
    if (s > 1) {
      if (tc_prec) {
        const int nkb_total = (int)(s / 64);
        const int waves = p->o.far_split > 0 ? p->o.far_split : 2;
        const int ks = far_ksplit(n_active, nkb_total, p->sms, waves);
        A.ksplit = 1;  // the K-split parts are added on the device
        if (ks > 1)  // split tiles add their parts; unsplit tiles store
          CK(cudaMemsetAsync(p->farb, 0, (size_t)n_active * 2 * B * kTrajPerTile * d * sizeof(double), st),
             "far sums reset");
        FarTcArgs T = far_tc_args(p, p->d_tiles, p->d_tmapF, s, n_active, ks);
        Trace tr(p, ABM_KERNEL_FAR, st);
        CK(launch_far_tc(far_kind(p), T, n_active, st), "tensor-core far kernel");
      } else {
        // history split of the SIMT far kernels per launch: about two CTAs per
        // SM over the active tiles (few tiles late in a ragged batch would
        // otherwise leave most SMs idle); the near kernel of this time tile
        // adds the same number of partial sums
        int ks = std::max(1, std::min(16, (2 * p->sms + n_active - 1) / n_active));
        while (ks > 1 && (size_t)ks * n_active * 2 * B * kTrajPerTile * d > p->farb_cap) --ks;
        A.ksplit = ks;
        {
          Trace tr(p, ABM_KERNEL_FAR, st);
          CK(launch_batched_far(d, p->o.prec, A, n_active, s, st), "far kernel");
        }
        A.ksplit = 1;  // the far kernel's last CTA per tile added the partials
      }
    }
    {
      Trace tr(p, ABM_KERNEL_NEAR, st);
      // warps per component: helpers hide the chain's latency when few tiles are
      // active; with many tiles per SM the tiles hide each other's and the
      // chain-only form needs fewer instructions
      const int wpc = p->o.near_warps ? p->o.near_warps
                                      : (n_active <= p->sms ? 3 : (n_active <= 2 * p->sms ? 2 : 1));
      // few active tiles: spread each over several CTAs so the FP64 window work
      // of the tail runs on more SMs.  Measured per step on GB300 (Rossler):
      // one CTA with helper warps 3.05 us, split 2 3.65 us, split 4 2.7 us,
      // split 8 2.35 us, so the automatic choice uses 4 or 8 only (taking 16
      // first where it fits changed the Rossler near time by 0.4 %: the tail's
      // steps are bound by the chain's latency, not by the SMs in use).
      int split = p->o.near_split;
      if (split == 0) {
        split = 1;
        for (int c : {8, 4})
          if ((long long)n_active * c <= p->sms) { split = c; break; }
      }
      CK(launch_batched_near(p->sys, A, n_active, s, B, wpc, split, st), "near kernel");
    }
    if (out && j < (int)out->ops.size() && !out->ops[j].empty()) {
      cudaEvent_t ev = p->hio_ev[j];
      CK(cudaEventRecord(ev, st), "event");
      CK(cudaStreamWaitEvent(p->copy_st, ev, 0), "event wait");
      const size_t hp = (size_t)out->ldh * d * sizeof(double), dp = (size_t)out->ldd * d * sizeof(double);
      for (const CopyOp& c : out->ops[j]) {
        const size_t width = (size_t)(c.hi - c.lo + 1) * d * sizeof(double);
        const size_t ho = ((size_t)c.i0 * out->ldh + c.lo) * d, dof = ((size_t)c.i0 * out->ldd + c.lo) * d;
        CK(cudaMemcpy2DAsync(out->Yh + ho, hp, out->Yd + dof, dp, width, c.n, cudaMemcpyDeviceToHost, p->copy_st),
           "copy-out");
        if (out->YPh)
          CK(cudaMemcpy2DAsync(out->YPh + ho, hp, out->YPd + dof, dp, width, c.n, cudaMemcpyDeviceToHost,
                               p->copy_st), "copy-out");
      }
    }
  }
  return ABM_OK;
}

// Kernel arguments of one batched solve (tables from schedule_batch).
BatchArgs batch_args(abm_plan p, const Sched& S, const double* params, const double* y0, const double* y0d,
                     double* Y, double* YP, long long ldY) {
  const int d = p->d;
  const size_t NT = (size_t)kMaxWeightSets * kMaxD;
  BatchArgs A{};
  A.tiles = p->d_tiles;
  A.n_tiles = S.n_tiles;
  A.B = p->B;
  A.ksplit = S.ksplit;
  A.far_k0 = 1;
  A.per_comp = S.per_comp ? 1 : 0;
  A.bucket_alpha = p->d_balpha;
  A.bucket_b = p->d_bptr;
  A.bucket_a = p->d_bptr + NT;
  A.bucket_c = p->d_bptr + 2 * NT;
  A.bucket_b32 = p->d_b32ptr;
  A.bucket_a32 = p->d_b32ptr + NT;
  A.bucket_g = p->d_bg;
  A.bucket_taylor = p->d_btaylor;
  A.h = p->d_h;
  A.N = p->d_N;
  A.params = params;
  A.y0 = y0;
  A.y0d = y0d;
  A.hhat = p->d_hhat;
  A.F = p->Fb;
  A.F32 = (p->o.prec == ABM_PREC_FP32_FAR) ? p->Fb32 : nullptr;
  A.Fsh = p->Fsh;
  A.fsh_ld = p->fsh_ld;
  A.fsh_plane = (long long)p->max_tiles * kTrajPerTile * d * p->fsh_ld;
  A.far = p->farb;
  A.far_ticket = p->far_ticket;
  A.Y = Y;
  A.YP = YP;
  A.ldY = ldY;
  A.status = p->status;
  A.passes = p->o.corrector_passes > 1 ? p->o.corrector_passes : 1;
  A.f_elems = (long long)p->fb_cap;
  A.w_elems = (long long)p->Mw + 1;
  A.far_elems = (long long)p->farb_cap;
  A.y_elems = (long long)S.M * ldY * d;
  A.fsh_plane_elems = A.fsh_plane;
  A.bad_traj = p->o.test_bad_index > 0 ? p->o.test_bad_index - 1 : -1;
  return A;
}

template <typename T>
void key_append(std::vector<unsigned char>& k, const T* v, size_t n) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(v);
  k.insert(k.end(), b, b + n * sizeof(T));
}

}  // namespace

extern "C" {

void abm_plan_opts_default(abm_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->prec = ABM_PREC_FP64;
}

int abm_system_dim(abm_system sys) { return sys_dim(sys); }
int abm_system_nparams(abm_system sys) { return sys_nparams(sys); }

const char* abm_last_error(abm_plan p) { return p ? p->err.c_str() : "null plan"; }

abm_status abm_plan_create(abm_plan* out, abm_system sys, const abm_plan_opts* o) {
  if (!out || !o) return ABM_ERR_INVALID_ARG;
  *out = nullptr;
  if (sys_dim(sys) < 0 || o->n_max < 1 || o->max_batch < 0 || o->tile_B < 0 || o->far_ctas < 0 ||
      o->spin_timeout_cycles < 0 || (o->prec != ABM_PREC_FP64 && o->prec != ABM_PREC_FP32_FAR &&
                                     o->prec != ABM_PREC_BF16X3_FAR && o->prec != ABM_PREC_BF16X6_FAR))
    return ABM_ERR_INVALID_ARG;
  for (int r : o->reserved)
    if (r) return ABM_ERR_INVALID_ARG;
  if (o->tile_B && o->tile_B != 64 && o->tile_B != 32) return ABM_ERR_UNSUPPORTED;
  if (o->near_warps != 0 && o->near_warps != 1 && o->near_warps != 2 && o->near_warps != 3 && o->near_warps != 5)
    return ABM_ERR_INVALID_ARG;
  if (o->far_split < 0 || o->far_split > 64) return ABM_ERR_INVALID_ARG;
  if (o->near_split != 0 && o->near_split != 1 && o->near_split != 2 && o->near_split != 4 && o->near_split != 8 &&
      o->near_split != 16)
    return ABM_ERR_INVALID_ARG;
  if (o->corrector_passes < 0 || o->corrector_passes > 8) return ABM_ERR_INVALID_ARG;
  if (o->test_bad_index < 0) return ABM_ERR_INVALID_ARG;
#ifndef ABM_CHECKED
  if (o->test_bad_index != 0) return ABM_ERR_UNSUPPORTED;  // only a checked build may offset an index
#endif
  const bool tc_prec = o->prec == ABM_PREC_BF16X3_FAR || o->prec == ABM_PREC_BF16X6_FAR;
  if (tc_prec && (sys_dim(sys) != 3 || (o->tile_B && o->tile_B != 64))) return ABM_ERR_UNSUPPORTED;
  abm_plan p = new abm_plan_s();
  p->sys = sys;
  p->d = sys_dim(sys);
  p->np = sys_nparams(sys);
  p->o = *o;
  p->B = o->tile_B ? o->tile_B : kDefaultB;
  p->wsets.resize(kMaxWeightSets);
  auto cleanup_fail = [&](abm_status s) { abm_plan_destroy(p); return s; };
  if (cudaGetDevice(&p->device) != cudaSuccess) return cleanup_fail(ABM_ERR_CUDA);
  if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    return cleanup_fail(ABM_ERR_CUDA);
  p->G = o->far_ctas ? o->far_ctas : p->sms;
  const int B = p->B, d = p->d;
  const long long rows = (long long)((o->n_max + B - 1) / B) * B + 1;  // tiles run whole
  p->Mw = (int)(rows + 2 * B + 2);
  auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, bytes) == cudaSuccess; };
  if (!alloc((void**)&p->status, sizeof(unsigned long long)) ||
      !alloc((void**)&p->F1, (size_t)(rows + B) * d * sizeof(double)) ||
      !alloc((void**)&p->far1, (size_t)2 * B * 2 * d * sizeof(double)) ||
      !alloc((void**)&p->part1, (size_t)2 * p->G * B * 2 * d * sizeof(double)) ||
      !alloc((void**)&p->tickets, 2 * sizeof(unsigned int)) ||
      !alloc((void**)&p->hhat1, sizeof(double)))
    return cleanup_fail(ABM_ERR_OOM);
  p->Gp = std::min(persistent_max_grid(sys), o->far_ctas ? o->far_ctas + 1 : p->sms);
  if (p->Gp < 2) return cleanup_fail(ABM_ERR_UNSUPPORTED);
  if (!alloc((void**)&p->ppartial, (size_t)kPersistRing * (p->Gp - 1) * kPersistB * 2 * d * sizeof(double)) ||
      !alloc((void**)&p->pflags, (1 + kPersistRing) * sizeof(unsigned long long)))
    return cleanup_fail(ABM_ERR_OOM);
  cudaMemset(p->status, 0, sizeof(unsigned long long));
  cudaMemset(p->tickets, 0, 2 * sizeof(unsigned int));
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess) return cleanup_fail(ABM_ERR_CUDA);
  for (int i = 0; i < kEventRing; ++i) {
    if (cudaEventCreateWithFlags(&p->ev_near[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_far[i], cudaEventDisableTiming) != cudaSuccess)
      return cleanup_fail(ABM_ERR_CUDA);
  }
  if (cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming) != cudaSuccess)
    return cleanup_fail(ABM_ERR_CUDA);
  if (o->max_batch > 0) {
    // every trajectory may sit in its own tile in the worst case of many alphas
    p->max_tiles = (o->max_batch + kTrajPerTile - 1) / kTrajPerTile + kMaxWeightSets;
    p->max_tiles = std::min(p->max_tiles, o->max_batch);
    p->fb_cap = (size_t)p->max_tiles * rows * kTrajPerTile * d;
    size_t far_units = 2 * (size_t)p->max_tiles + 2 * (size_t)p->sms + 16;  // adjoint: 2 tiles per tile
    p->farb_cap = far_units * 2 * B * kTrajPerTile * d;
    if (!alloc((void**)&p->Fb, p->fb_cap * sizeof(double)) ||
        (o->prec == ABM_PREC_FP32_FAR && !alloc((void**)&p->Fb32, p->fb_cap * sizeof(float))) ||
        !alloc((void**)&p->farb, p->farb_cap * sizeof(double)) ||
        !alloc((void**)&p->far_ticket, (2 * (size_t)p->max_tiles + 16) * sizeof(unsigned int)) ||
        !alloc((void**)&p->d_tiles, (size_t)p->max_tiles * sizeof(TileDesc)) ||
        !alloc((void**)&p->d_h, (size_t)o->max_batch * sizeof(double)) ||
        !alloc((void**)&p->d_N, (size_t)o->max_batch * sizeof(int)) ||
        !alloc((void**)&p->d_hhat, (size_t)o->max_batch * kMaxD * sizeof(double)) ||
        !alloc((void**)&p->d_balpha, kMaxWeightSets * kMaxD * sizeof(double)) ||
        !alloc((void**)&p->d_bg, kMaxWeightSets * kMaxD * sizeof(double)) ||
        !alloc((void**)&p->d_btaylor, kMaxWeightSets * sizeof(int)) ||
        !alloc((void**)&p->d_bptr, 3 * kMaxWeightSets * kMaxD * sizeof(double*)) ||
        !alloc((void**)&p->d_b32ptr, 2 * kMaxWeightSets * kMaxD * sizeof(float*)))
      return cleanup_fail(ABM_ERR_OOM);
    if (cudaMemset(p->far_ticket, 0, (2 * (size_t)p->max_tiles + 16) * sizeof(unsigned int)) != cudaSuccess)
      return cleanup_fail(ABM_ERR_CUDA);
    if (tc_prec) {
      p->Lbase = (long long)((o->n_max + 63) / 64) * 64;
      p->Lx = p->Lbase + 64;
      p->fsh_ld = p->Lbase + 64;
      const size_t gcols = (size_t)p->max_tiles * kTrajPerTile * d;
      if (!alloc((void**)&p->Fsh, 3 * gcols * p->fsh_ld * sizeof(__nv_bfloat16)) ||
          !alloc((void**)&p->d_tmapW, (size_t)kMaxWeightSets * 3 * sizeof(CUtensorMap)) ||
          !alloc((void**)&p->d_tmapF, 3 * sizeof(CUtensorMap)))
        return cleanup_fail(ABM_ERR_OOM);
      CUtensorMap mf[3];
      for (int q = 0; q < 3; ++q)
        if (!make_tmap_bf16(&mf[q], p->Fsh + (size_t)q * gcols * p->fsh_ld, 64, gcols * (p->fsh_ld / 64),
                            (unsigned)(kTrajPerTile * d)))
          return cleanup_fail(ABM_ERR_CUDA);
      if (cudaMemcpy(p->d_tmapF, mf, sizeof(mf), cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup_fail(ABM_ERR_CUDA);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return cleanup_fail(ABM_ERR_CUDA);
  *out = p;
  return ABM_OK;
}

abm_status abm_plan_destroy(abm_plan p) {
  if (!p) return ABM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  for (auto& w : p->wsets) {
    cudaFree(w.b); cudaFree(w.a); cudaFree(w.c); cudaFree(w.g); cudaFree(w.b32); cudaFree(w.a32); cudaFree(w.Wx);
  }
  cudaFree(p->Fsh); cudaFree(p->d_tmapW); cudaFree(p->d_tmapF); 
  cudaFree(p->Xadj); cudaFree(p->Xsh); cudaFree(p->d_tmapX); cudaFree(p->d_atiles);
  cudaFree(p->acc_dp); cudaFree(p->acc_dy0); cudaFree(p->phi0c);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  cudaFree(p->hio_params); cudaFree(p->hio_y0); cudaFree(p->hio_Y); cudaFree(p->hio_YP);
  cudaFree(p->hio_Y1); cudaFree(p->hio_YP1);
  for (cudaEvent_t e : p->hio_ev) cudaEventDestroy(e);
  if (p->hio_done) cudaEventDestroy(p->hio_done);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  cudaFree(p->ppartial); cudaFree(p->pflags);
  cudaFree(p->F1); cudaFree(p->far1); cudaFree(p->part1); cudaFree(p->tickets); cudaFree(p->hhat1);
  cudaFree(p->Fb); cudaFree(p->Fb32); cudaFree(p->farb); cudaFree(p->far_ticket); cudaFree(p->d_tiles); cudaFree(p->d_h);
  cudaFree(p->d_N); cudaFree(p->d_hhat); cudaFree(p->d_balpha); cudaFree(p->d_bg);
  cudaFree(p->d_bptr); cudaFree(p->d_b32ptr); cudaFree(p->d_btaylor); cudaFree(p->status);
  if (p->side) cudaStreamDestroy(p->side);
  for (int i = 0; i < kEventRing; ++i) {
    if (p->ev_near[i]) cudaEventDestroy(p->ev_near[i]);
    if (p->ev_far[i]) cudaEventDestroy(p->ev_far[i]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  for (auto& e : p->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  delete p;
  return ABM_OK;
}

abm_status abm_plan_sync(abm_plan p, void* stream, int64_t* where) {
  if (!p) return ABM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(st), "stream synchronize");
  unsigned long long w = 0;
  CK(cudaMemcpy(&w, p->status, sizeof(w), cudaMemcpyDeviceToHost), "status read");
  if (w) CK(cudaMemset(p->status, 0, sizeof(w)), "status clear");
  int code = (int)(w >> 60);
  if (where) *where = (int64_t)(w & 0x0FFFFFFFFFFFFFFFull);
  if (code == 0) return ABM_OK;
  char buf[200];
  status_text(w, buf, sizeof buf);
  return fail(p, (abm_status)code, std::string("device reported ") + buf);
}

abm_status abm_weights(abm_plan p, double alpha, int M, double* b, double* a, double* c, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!order_ok(alpha) || M < 0 || !b || !a || !c)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_weights: alpha must be in (0,2], M >= 0, arrays non-null");
  CK(launch_weights(alpha, M, b, a, c, nullptr, (cudaStream_t)stream), "weights kernel");
  return ABM_OK;
}

abm_status abm_far_history(abm_plan p, double alpha, const double* F, long long rows, long long cols,
                           long long s, int B, long long k_lo, long long k_hi, double* P, double* C,
                           void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!alpha_ok(alpha) || !F || !P || !C || rows < 1 || (cols != 1 && cols != 3 && !p->Fsh) || B != p->B ||
      k_lo < 1 || k_hi < k_lo || k_hi > s || s >= rows || s + B > p->Mw - 2 * p->B)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_far_history: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  if (p->Fsh) return far_history_tc(p, alpha, F, rows, cols, s, B, k_lo, k_hi, P, C, st);
  if (p->o.prec != ABM_PREC_FP64) return fail(p, ABM_ERR_UNSUPPORTED, "abm_far_history: FP64 or tensor-core plans only");
  WeightSet* w;
  abm_status rs = get_weights(p, alpha, st, &w);
  if (rs) return rs;
  const int d = (int)cols;
  std::vector<double> zero;
  if (k_hi == k_lo) {
    CK(cudaMemsetAsync(P, 0, sizeof(double) * B * d, st), "memset");
    CK(cudaMemsetAsync(C, 0, sizeof(double) * B * d, st), "memset");
    return ABM_OK;
  }
  long long K = k_hi - k_lo;
  int grid = (int)std::min<long long>(p->G, (K + 63) / 64);
  FarSingleArgs A{F, w->b, w->a, s, k_lo, k_hi, (K + grid - 1) / grid, p->part1, p->far1, p->tickets};
  CK(launch_far_single(d, A, B, grid, st), "far kernel");
  // de-interleave [B][2d] into P and C
  CK(cudaMemcpy2DAsync(P, d * sizeof(double), p->far1, 2 * d * sizeof(double), d * sizeof(double), B,
                       cudaMemcpyDeviceToDevice, st), "copy P");
  CK(cudaMemcpy2DAsync(C, d * sizeof(double), p->far1 + d, 2 * d * sizeof(double), d * sizeof(double), B,
                       cudaMemcpyDeviceToDevice, st), "copy C");
  return ABM_OK;
}

}  // extern "C"

namespace {

// The single-trajectory solve behind abm_solve and abm_solve_ext: alpha holds
// one order per component (in (0, 2]); y0d the initial derivatives (NULL:
// zero), used by components of order above one.
// n0 > 0 (resume): F_in holds f_0..f_n0 of an earlier solve of the same
// problem (host or device memory); stepping restarts at the time tile that
// holds step n0 + 1, whose start row s0 <= n0 comes from F_in.
abm_status solve_single(abm_plan p, const char* who, const double* alpha, double h, int N, const double* params,
                        const double* y0, const double* y0d, double* Y, double* YP, cudaStream_t st,
                        int n0 = 0, const double* F_in = nullptr) {
  TrajParams tp{};
  for (int i = 0; i < p->np; ++i) {
    if (!std::isfinite(params[i])) return fail(p, ABM_ERR_INVALID_ARG, std::string(who) + ": non-finite parameter");
    tp.p[i] = params[i];
  }
  int taylor_mask = 0;
  for (int i = 0; i < p->d; ++i) {
    if (!std::isfinite(y0[i]) || (y0d && !std::isfinite(y0d[i])))
      return fail(p, ABM_ERR_INVALID_ARG, std::string(who) + ": non-finite y0 or y0d");
    tp.y0[i] = y0[i];
    if (alpha[i] > 1.0) {
      taylor_mask |= 1 << i;
      tp.y0d[i] = y0d ? y0d[i] : 0.0;
    }
  }
  // one weight set per distinct order
  PersistArgs A{};
  int nc = 1;
  for (int i = 0; i < p->d; ++i) {
    if (alpha[i] != alpha[0]) nc = p->d;
    int same = -1;
    for (int j = 0; j < i && same < 0; ++j)
      if (alpha[j] == alpha[i]) same = j;
    if (same >= 0) {
      A.b[i] = A.b[same];
      A.a[i] = A.a[same];
      A.c[i] = A.c[same];
      A.g[i] = A.g[same];
      continue;
    }
    WeightSet* w = nullptr;  // the least recently used set is reused: never one taken above
    abm_status rs = get_weights(p, alpha[i], st, &w);
    if (rs) return rs;
    A.b[i] = w->b;
    A.a[i] = w->a;
    A.c[i] = w->c;
    A.g[i] = w->g;
  }
  // one cooperative launch: CTA 0 steps, CTAs 1..Gp-1 compute the far history
  CK(cudaMemsetAsync(p->pflags, 0, (1 + kPersistRing) * sizeof(unsigned long long), st), "flags reset");
  A.F = p->F1;
  A.Y = Y;
  A.YP = YP;
  A.partial = p->ppartial;
  A.flags = p->pflags;
  A.status = p->status;
  A.tp = tp;
  for (int i = 0; i < kMaxD; ++i) A.alpha[i] = alpha[i < p->d ? i : 0];
  A.h = h;
  A.taylor_mask = taylor_mask;
  A.N = N;
  A.spin_budget = p->o.spin_timeout_cycles > 0 ? p->o.spin_timeout_cycles : 4000000000LL;
  A.withhold_tile = p->o.test_withhold_tile > 0 ? p->o.test_withhold_tile - 1 : -1;
  A.passes = p->o.corrector_passes > 1 ? p->o.corrector_passes : 1;
  A.start_tile = n0 / kPersistB;
  A.f_elems = (long long)(((p->o.n_max + p->B - 1) / p->B) * p->B + 1 + p->B) * p->d;
  A.w_elems = (long long)p->Mw + 1;
  A.partial_elems = (long long)kPersistRing * (p->Gp - 1) * kPersistB * 2 * p->d;
  if (A.start_tile > 0)
    CK(cudaMemcpyAsync(p->F1, F_in, (size_t)(A.start_tile * kPersistB + 1) * p->d * sizeof(double),
                       cudaMemcpyDefault, st), "history import");
  {
    Trace tr(p, ABM_KERNEL_SINGLE, st);
    CK(launch_persistent(p->sys, nc, A, p->Gp, st), "persistent single-trajectory kernel");
  }
  p->last_single_rows = N + 1;
  return ABM_OK;
}

}  // namespace

extern "C" {

abm_status abm_solve(abm_plan p, double alpha, double h, int N, const double* params, const double* y0,
                     double* Y, double* YP, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!alpha_ok(alpha) || !(std::isfinite(h) && h > 0.0) || N < 1 || N > p->o.n_max || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve: need alpha in (0,1], finite h > 0, 1 <= N <= n_max, "
                                        "non-null params/y0/Y");
  const double al[kMaxD] = {alpha, alpha, alpha};
  return solve_single(p, "abm_solve", al, h, N, params, y0, nullptr, Y, YP, (cudaStream_t)stream);
}

abm_status abm_solve_ext(abm_plan p, const double* alpha, double h, int N, const double* params, const double* y0,
                         const double* y0d, double* Y, double* YP, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!alpha || !(std::isfinite(h) && h > 0.0) || N < 1 || N > p->o.n_max || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_ext: need finite h > 0, 1 <= N <= n_max, "
                                        "non-null alpha/params/y0/Y");
  for (int i = 0; i < p->d; ++i)
    if (!order_ok(alpha[i])) return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_ext: every order must be in (0, 2]");
  return solve_single(p, "abm_solve_ext", alpha, h, N, params, y0, y0d, Y, YP, (cudaStream_t)stream);
}

abm_status abm_solve_host(abm_plan p, double alpha, double h, int N, const double* params, const double* y0,
                          double* Y, double* YP, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!alpha_ok(alpha) || !(std::isfinite(h) && h > 0.0) || N < 1 || N > p->o.n_max || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_host: need alpha in (0,1], finite h > 0, 1 <= N <= n_max, "
                                        "non-null params/y0/Y");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)(N + 1) * p->d * sizeof(double);
  const size_t cap = (size_t)(p->o.n_max + 1) * p->d * sizeof(double);
  if (!p->hio_Y1) CK(cudaMalloc(&p->hio_Y1, cap), "host-io Y");
  if (YP && !p->hio_YP1) CK(cudaMalloc(&p->hio_YP1, cap), "host-io YP");
  const double al[kMaxD] = {alpha, alpha, alpha};
  abm_status rs = solve_single(p, "abm_solve_host", al, h, N, params, y0, nullptr, p->hio_Y1, YP ? p->hio_YP1 : nullptr,
                               st);
  if (rs) return rs;
  CK(cudaMemcpyAsync(Y, p->hio_Y1, bytes, cudaMemcpyDeviceToHost, st), "copy-out");
  if (YP) CK(cudaMemcpyAsync(YP, p->hio_YP1, bytes, cudaMemcpyDeviceToHost, st), "copy-out");
  return ABM_OK;
}

abm_status abm_history(abm_plan p, int rows, double* F, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!F || rows < 1 || rows > p->last_single_rows)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_history: need 1 <= rows <= N+1 of the last single-trajectory solve "
                                        "and a non-null F");
  CK(cudaMemcpyAsync(F, p->F1, (size_t)rows * p->d * sizeof(double), cudaMemcpyDefault, (cudaStream_t)stream),
     "history export");
  return ABM_OK;
}

abm_status abm_solve_resume(abm_plan p, const double* alpha, double h, int n0, int N, const double* params,
                            const double* y0, const double* y0d, const double* F, double* Y, double* YP,
                            void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (!alpha || !(std::isfinite(h) && h > 0.0) || N < 1 || N > p->o.n_max || n0 < 0 || n0 > N || !params || !y0 ||
      !Y || (n0 >= kPersistB && !F))
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_resume: need finite h > 0, 0 <= n0 <= N <= n_max, "
                                        "non-null alpha/params/y0/Y and the history F");
  for (int i = 0; i < p->d; ++i)
    if (!order_ok(alpha[i])) return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_resume: every order must be in (0, 2]");
  if (n0 == N) return ABM_OK;
  return solve_single(p, "abm_solve_resume", alpha, h, N, params, y0, y0d, Y, YP, (cudaStream_t)stream, n0, F);
}

}  // extern "C"

namespace {

// abm_solve_batched / abm_solve_batched_ext: alpha holds M orders (astride 1)
// or M x d (astride d), y0d the initial derivatives (device, may be null).
abm_status solve_batched_impl(abm_plan p, const char* who, int M, const double* alpha, int astride, double amax,
                              const double* h, const int* N, const double* params, const double* y0,
                              const double* y0d, double* Y, long long ldY, double* YP, cudaStream_t st) {
  // with use_graph, a call whose arguments equal those of the captured call
  // replays the graph (the device tables it reads are still in place)
  std::vector<unsigned char> key;
  if (p->o.use_graph) {
    key_append(key, &M, 1);
    key_append(key, &astride, 1);
    key_append(key, alpha, (size_t)M * astride);
    key_append(key, h, M);
    key_append(key, N, M);
    const void* ptrs[5] = {params, y0, Y, YP, y0d};
    key_append(key, ptrs, 5);
    key_append(key, &ldY, 1);
    if (p->graph_exec && key == p->graph_key) {
      CK(cudaGraphLaunch(p->graph_exec, st), "graph launch");  // the key fixes every value checked before
      return ABM_OK;
    }
  }
  Sched S;
  abm_status rs = schedule_batch(p, M, alpha, astride, amax, h, N, ldY, st, S, who);
  if (rs) return rs;
  const BatchArgs A = batch_args(p, S, params, y0, y0d, Y, YP, ldY);
  if (!p->o.use_graph) return enqueue_batched(p, S, A, st);
  // capture the launch sequence on the plan's side stream, after the uploads
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  CK(cudaEventRecord(p->ev_start, st), "event");
  CK(cudaStreamWaitEvent(p->side, p->ev_start, 0), "event wait");
  CK(cudaStreamBeginCapture(p->side, cudaStreamCaptureModeThreadLocal), "begin capture");
  p->capturing = true;
  rs = enqueue_batched(p, S, A, p->side);
  p->capturing = false;
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(p->side, &graph);
  if (rs) { if (graph) cudaGraphDestroy(graph); return rs; }
  if (ce != cudaSuccess) return cuda_fail(p, ce, "end capture");
  ce = cudaGraphInstantiate(&p->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) { p->graph_exec = nullptr; return cuda_fail(p, ce, "graph instantiate"); }
  p->graph_key = key;
  CK(cudaGraphLaunch(p->graph_exec, st), "graph launch");
  return ABM_OK;
}

}  // namespace

extern "C" {

abm_status abm_solve_batched(abm_plan p, int M, const double* alpha, const double* h, const int* N,
                             const double* params, const double* y0, double* Y, long long ldY, double* YP,
                             void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_batched: need 1 <= M <= max_batch and non-null arrays");
  return solve_batched_impl(p, "abm_solve_batched", M, alpha, 1, 1.0, h, N, params, y0, nullptr, Y, ldY, YP,
                            (cudaStream_t)stream);
}

abm_status abm_solve_batched_ext(abm_plan p, int M, const double* alpha, const double* h, const int* N,
                                 const double* params, const double* y0, const double* y0d, double* Y,
                                 long long ldY, double* YP, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_batched_ext: need 1 <= M <= max_batch and non-null arrays");
  return solve_batched_impl(p, "abm_solve_batched_ext", M, alpha, p->d, 2.0, h, N, params, y0, y0d, Y, ldY, YP,
                            (cudaStream_t)stream);
}

abm_status abm_history_batched(abm_plan p, int M, const double* alpha, const double* h, const int* N, int rows,
                               double* F, long long ldF, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !F || rows < 1 || ldF < rows)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_history_batched: need 1 <= M <= max_batch, rows >= 1, ldF >= rows "
                                        "and non-null arrays");
  cudaStream_t st = (cudaStream_t)stream;
  int nmax = 0;  // the output has no ldY: the schedule is checked against the longest trajectory
  for (int i = 0; i < M; ++i) nmax = std::max(nmax, N[i]);
  Sched S;
  abm_status rs = schedule_batch(p, M, alpha, p->d, 2.0, h, N, (long long)nmax + 1, st, S, "abm_history_batched");
  if (rs) return rs;
  const BatchArgs A = batch_args(p, S, nullptr, nullptr, nullptr, nullptr, nullptr, S.nmax + 1);
  CK(launch_export_history(p->d, A, S.n_tiles, std::min<long long>(rows, (long long)S.nmax + 1), F, ldF,
                           (long long)M * ldF * p->d, st),
     "history export kernel");
  return ABM_OK;
}

abm_status abm_solve_batched_resume(abm_plan p, int M, const double* alpha, const double* h, const int* N, int n0,
                                    const double* params, const double* y0, const double* y0d, const double* F,
                                    long long ldF, double* Y, long long ldY, double* YP, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !params || !y0 || !Y || n0 < 0 ||
      (n0 >= p->B && (!F || ldF < (long long)n0 + 1)))
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_batched_resume: need 1 <= M <= max_batch, n0 >= 0, the history F "
                                        "with ldF >= n0 + 1 and non-null arrays");
  for (int i = 0; i < M; ++i)
    if (N[i] < n0) return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_batched_resume: every N[i] must be >= n0");
  cudaStream_t st = (cudaStream_t)stream;
  Sched S;
  abm_status rs = schedule_batch(p, M, alpha, p->d, 2.0, h, N, ldY, st, S, "abm_solve_batched_resume");
  if (rs) return rs;
  BatchArgs A = batch_args(p, S, params, y0, y0d, Y, YP, ldY);
  A.y_elems = (long long)M * ldY * p->d;
  A.resume_row = (long long)(n0 / p->B) * p->B;
  if (A.resume_row > 0)
    CK(launch_import_history(p->d, A, S.n_tiles, A.resume_row, F, ldF, (long long)M * ldF * p->d, st),
       "history import kernel");
  return enqueue_batched(p, S, A, st);
}

abm_status abm_solve_batched_host(abm_plan p, int M, const double* alpha, const double* h, const int* N,
                                  const double* params, const double* y0, double* Y, long long ldY, double* YP,
                                  void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !params || !y0 || !Y)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_solve_batched_host: need 1 <= M <= max_batch and non-null arrays");
  cudaStream_t st = (cudaStream_t)stream;
  const int d = p->d, B = p->B;
  const long long ldd = (long long)p->o.n_max + 1;  // leading dimension of the device copy of Y
  // device buffers and the copy stream, once per plan
  if (!p->hio_Y) {
    CK(cudaMalloc(&p->hio_params, (size_t)p->o.max_batch * std::max(1, p->np) * sizeof(double)), "host-io params");
    CK(cudaMalloc(&p->hio_y0, (size_t)p->o.max_batch * d * sizeof(double)), "host-io y0");
    CK(cudaMalloc(&p->hio_Y, (size_t)p->o.max_batch * ldd * d * sizeof(double)), "host-io Y");
    CK(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking), "copy stream");
    CK(cudaEventCreateWithFlags(&p->hio_done, cudaEventDisableTiming), "event");
  }
  if (YP && !p->hio_YP) CK(cudaMalloc(&p->hio_YP, (size_t)p->o.max_batch * ldd * d * sizeof(double)), "host-io YP");
  Sched S;
  abm_status rs = schedule_batch(p, M, alpha, 1, 1.0, h, N, ldY, st, S, "abm_solve_batched_host");
  if (rs) return rs;
  // inputs up, then the solve with finished rows copied out behind the time
  // tiles that complete them
  CK(cudaMemcpyAsync(p->hio_params, params, (size_t)M * p->np * sizeof(double), cudaMemcpyHostToDevice, st),
     "params upload");
  CK(cudaMemcpyAsync(p->hio_y0, y0, (size_t)M * d * sizeof(double), cudaMemcpyHostToDevice, st), "y0 upload");
  HostCopyOut out;
  out.ops = plan_copy_out(M, N, B, (S.nmax + B - 1) / B);
  while (p->hio_ev.size() < out.ops.size()) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    p->hio_ev.push_back(e);
  }
  out.Yh = Y;
  out.YPh = YP;
  out.ldh = ldY;
  out.Yd = p->hio_Y;
  out.YPd = YP ? p->hio_YP : nullptr;
  out.ldd = ldd;
  const BatchArgs A = batch_args(p, S, p->hio_params, p->hio_y0, nullptr, p->hio_Y, YP ? p->hio_YP : nullptr, ldd);
  rs = enqueue_batched(p, S, A, st, &out);
  if (rs) return rs;
  CK(cudaEventRecord(p->hio_done, p->copy_st), "event");
  CK(cudaStreamWaitEvent(st, p->hio_done, 0), "event wait");  // the call's work ends on st
  return ABM_OK;
}

abm_status abm_plan_kernel_times(abm_plan p, abm_kernel_kind kind, void* stream, int reset, long long* launches,
                                 double* total_ms) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if ((int)kind < 0 || (int)kind >= ABM_KERNEL_KINDS) return fail(p, ABM_ERR_INVALID_ARG, "unknown kernel kind");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  CK(cudaDeviceSynchronize(), "device synchronize");
  double ms = 0.0;
  std::vector<std::pair<int, size_t>> keep;
  for (auto& u : p->ev_used) {
    if (u.first != (int)kind) { keep.push_back(u); continue; }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev_pool[u.second].first, p->ev_pool[u.second].second) == cudaSuccess) ms += t;
    if (!reset) keep.push_back(u);
  }
  if (launches) *launches = p->launches[kind];
  if (total_ms) *total_ms = ms;
  if (reset) {
    p->launches[kind] = 0;
    // event pairs of the reset kind become free again: rebuild the used list
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
    std::vector<std::pair<int, size_t>> used;
    std::vector<bool> taken(p->ev_pool.size(), false);
    for (auto& u : keep) {
      used.push_back({u.first, pool.size()});
      pool.push_back(p->ev_pool[u.second]);
      taken[u.second] = true;
    }
    for (size_t i = 0; i < p->ev_pool.size(); ++i)
      if (!taken[i]) pool.push_back(p->ev_pool[i]);
    p->ev_pool.swap(pool);
    p->ev_used.swap(used);
  }
  return ABM_OK;
}

abm_status abm_adjoint(abm_plan p, int M, const double* alpha, const double* h, const int* N, const double* params,
                       const double* y0, const double* Y, const double* YP, long long ldY, const double* dLdY,
                       double* dparams, double* dy0, void* stream) {
  if (!p) return ABM_ERR_INVALID_ARG;
  if (M < 1 || M > p->o.max_batch || !alpha || !h || !N || !params || !y0 || !Y || !YP || !dLdY || !dparams || !dy0)
    return fail(p, ABM_ERR_INVALID_ARG, "abm_adjoint: need 1 <= M <= max_batch and non-null arrays (Y and YP too)");
  if (p->o.prec == ABM_PREC_FP32_FAR)
    return fail(p, ABM_ERR_UNSUPPORTED, "abm_adjoint: FP64 or tensor-core (BF16X3/X6) plans only");
  if (p->o.corrector_passes > 1)
    return fail(p, ABM_ERR_UNSUPPORTED, "abm_adjoint: the adjoint of PECE only (corrector_passes <= 1)");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = p->B, d = p->d;
  Sched S;
  abm_status rs = schedule_batch(p, M, alpha, 1, 1.0, h, N, ldY, st, S, "abm_adjoint");
  if (rs) return rs;
  const int n_tiles = S.n_tiles;
  const bool tc_prec = p->Fsh != nullptr;
  // ---- adjoint workspace ----
  const size_t gcols = (size_t)2 * p->max_tiles * kTrajPerTile * d;
  if (!p->Xadj) {
    CK(cudaMalloc(&p->Xadj, 2 * p->fb_cap * sizeof(double)), "adjoint histories");
    CK(cudaMalloc(&p->d_atiles, (size_t)2 * p->max_tiles * sizeof(TileDesc)), "adjoint tiles");
    CK(cudaMalloc(&p->acc_dp, (size_t)p->o.max_batch * kMaxD * kMaxParams * sizeof(double)), "adjoint sums");
    CK(cudaMalloc(&p->acc_dy0, (size_t)p->o.max_batch * kMaxD * sizeof(double)), "adjoint sums");
    CK(cudaMalloc(&p->phi0c, (size_t)p->o.max_batch * kMaxD * sizeof(double)), "adjoint sums");
    if (tc_prec) {
      CK(cudaMalloc(&p->Xsh, 3 * gcols * p->fsh_ld * sizeof(__nv_bfloat16)), "adjoint planes");
      CK(cudaMalloc(&p->d_tmapX, 3 * sizeof(CUtensorMap)), "adjoint tensor maps");
      CUtensorMap mx[3];
      for (int q = 0; q < 3; ++q)
        if (!make_tmap_bf16(&mx[q], p->Xsh + (size_t)q * gcols * p->fsh_ld, 64, gcols * (p->fsh_ld / 64),
                            (unsigned)(kTrajPerTile * d)))
          return fail(p, ABM_ERR_CUDA, "abm_adjoint: tensor map of the adjoint planes");
      CK(cudaMemcpy(p->d_tmapX, mx, sizeof(mx), cudaMemcpyHostToDevice), "adjoint tensor maps");
    }
  }
  // two adjoint tiles (mu~, lambda~) per forward tile, same trajectories and group
  std::vector<TileDesc> at(2 * n_tiles);
  size_t off = 0;
  for (int t = 0; t < n_tiles; ++t) {
    const long long rows = (long long)((S.tiles[t].n_tile + B - 1) / B) * B + 1;
    for (int hh = 0; hh < 2; ++hh) {
      at[2 * t + hh] = S.tiles[t];
      at[2 * t + hh].slot = 2 * t + hh;  // the adjoint histories' pieces, tile 2t + hist
      at[2 * t + hh].f_off = (long long)off;
      off += (size_t)rows * kTrajPerTile * d;
    }
  }
  CK(cudaMemcpyAsync(p->d_atiles, at.data(), at.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, st), "adjoint tiles");
  AdjArgs A{};
  A.tiles = p->d_tiles;
  A.atiles = p->d_atiles;
  A.B = p->B;
  A.bucket_alpha = p->d_balpha;
  A.bucket_b = p->d_bptr;
  A.bucket_a = p->d_bptr + (size_t)kMaxWeightSets * kMaxD;
  A.bucket_c = p->d_bptr + 2 * (size_t)kMaxWeightSets * kMaxD;
  A.bucket_g = p->d_bg;
  A.h = p->d_h;
  A.N = p->d_N;
  A.params = params;
  A.y0 = y0;
  A.hhat = p->d_hhat;
  A.Y = Y;
  A.YP = YP;
  A.G = dLdY;
  A.ldY = ldY;
  A.X = p->Xadj;
  A.Xsh = p->Xsh;
  A.xsh_ld = p->fsh_ld;
  A.xsh_plane = (long long)gcols * p->fsh_ld;
  A.far = p->farb;
  A.acc_dp = p->acc_dp;
  A.acc_dy0 = p->acc_dy0;
  A.phi0c = p->phi0c;
  A.dparams = dparams;
  A.dy0 = dy0;
  A.status = p->status;
  {
    Trace tr(p, ABM_KERNEL_ADJOINT, st);
    CK(launch_adjoint_setup(p->sys, A, n_tiles, st), "adjoint setup kernel");
  }
  // FP64 far sums of the adjoint histories reuse the batched FP64 far kernel
  BatchArgs F{};
  F.tiles = p->d_atiles;
  F.B = B;
  F.far_k0 = 0;  // reversed row 0 (the k = N terms) is an ordinary row here
  F.bucket_alpha = p->d_balpha;
  F.bucket_b = p->d_bptr;
  F.bucket_a = p->d_bptr + (size_t)kMaxWeightSets * kMaxD;
  F.bucket_c = p->d_bptr + 2 * (size_t)kMaxWeightSets * kMaxD;
  F.bucket_g = p->d_bg;
  F.bucket_taylor = p->d_btaylor;
  F.F = p->Xadj;
  F.far = p->farb;
  F.far_ticket = p->far_ticket;
  F.status = p->status;
  F.f_elems = 2 * (long long)p->fb_cap;
  F.w_elems = (long long)p->Mw + 1;
  F.far_elems = (long long)p->farb_cap;
  F.bad_traj = -1;
  const int ntime = (S.nmax + B - 1) / B;
  int n_active = n_tiles;
  for (int j = 0; j < ntime; ++j) {
    const long long s = (long long)j * B;
    while (n_active > 0 && S.tiles[n_active - 1].n_tile <= s) --n_active;
    if (n_active == 0) break;
    const int na2 = 2 * n_active;
    A.far_tiles = na2;
    A.far_ksplit = 1;
    if (s > 0) {
      if (tc_prec) {
        const int nkb_total = (int)(s / 64);
        const int ks = far_ksplit(na2, nkb_total, p->sms, p->o.far_split > 0 ? p->o.far_split : 2);
        if (ks > 1)
          CK(cudaMemsetAsync(p->farb, 0, (size_t)na2 * 2 * B * kTrajPerTile * d * sizeof(double), st),
             "far sums reset");
        FarTcArgs T = far_tc_args(p, p->d_atiles, p->d_tmapX, s, na2, ks);
        Trace tr(p, ABM_KERNEL_ADJOINT, st);
        CK(launch_far_tc(far_kind(p), T, na2, st), "adjoint tensor-core far kernel");
      } else {
        int ks = std::max(1, std::min(16, (2 * p->sms + na2 - 1) / na2));
        while ((size_t)ks * na2 * 2 * B * kTrajPerTile * d > p->farb_cap && ks > 1) --ks;
        F.n_tiles = na2;
        F.ksplit = ks;
        A.far_ksplit = 1;  // the far kernel's last CTA per tile adds the ks partials
        Trace tr(p, ABM_KERNEL_ADJOINT, st);
        CK(launch_batched_far(d, ABM_PREC_FP64, F, na2, s, st), "adjoint far kernel");
      }
    }
    Trace tr(p, ABM_KERNEL_ADJOINT, st);
    // warps per component as in the forward near kernel (5 is not built here)
    const int wpc = p->o.near_warps ? std::min(p->o.near_warps, 3)
                                    : (n_active <= p->sms ? 3 : (n_active <= 2 * p->sms ? 2 : 1));
    // few active tiles: spread each over 4 or 8 CTAs as in the forward solve
    // (the adjoint split kernel is built for 4 and 8 only; 16 runs as 8)
    int split = p->o.near_split == 4 || p->o.near_split == 8 ? p->o.near_split : (p->o.near_split == 16 ? 8 : 1);
    if (p->o.near_split == 0)
      for (int c : {8, 4})
        if ((long long)n_active * c <= p->sms) { split = c; break; }
    CK(launch_adjoint_near(p->sys, A, n_active, s, B, wpc, split, st), "adjoint near kernel");
  }
  {
    Trace tr(p, ABM_KERNEL_ADJOINT, st);
    CK(launch_adjoint_finish(p->sys, A, M, st), "adjoint finish kernel");
  }
  return ABM_OK;
}

}  // extern "C"
