// A2 on the tensor cores: far-history Toeplitz-tile x F-tile contraction for
// the batched path, tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation
// in TMEM) fed by TMA, with the split-precision products of A5.
//
// For column tile t (32 trajectories x d components = 96 columns) and time
// tile s (targets n = s..s+63), the far sums of Sec. 2 over history rows
// k in [0, s) are one GEMM
//     D[128 x 96] = W[128 x s] * F[s x 96]
// with W rows 0..63 the predictor weights b_{s+i-k} (eq. (2)) and rows 64..127
// the corrector weights a_{s+i-k}, stacked so that both share one F tile.
// Row k = 0 of the BF16 history is kept zero: the j = 0 terms (b_n f_0,
// c_n f_0) are added in FP64 by the near kernel.
//
// Operands in HBM, both K-major so that a TMA box lands in the 128-byte
// swizzled layout the MMA reads, and K-block tiled: the 64 K values of one
// row and K block are 128 contiguous bytes, and the rows of one K block are
// contiguous, so every TMA box is a single contiguous read of 12-16 KB
// (a row-major K-major layout scatters each box over 96-128 rows of HBM).
//   W: "pre-expanded" Toeplitz, piece p of w_r(Lbase - x + r%64) at
//      ((x / 64) * 128 + r) * 64 + x % 64, so the tile of time tile s and
//      history block k0 is the block x = Lbase - s + k0 (a Toeplitz tile is a
//      shifted window of one vector; storing 128 shifted copies turns it into
//      a regular 2D tile).
//   F: history pieces, block (t, k / 64) = [96 columns][64 rows], written by
//      the near kernel at the end of each time tile.
// Split precision: x = x_hi + x_mid + x_lo, each BF16 (successive residuals).
//   kind 3 (BF16x3): hi*hi + hi*mid + mid*hi
//   kind 6 (BF16x6): + hi*lo + mid*mid + lo*hi (FP32-level error)
// The leading product hi*hi and the correction products accumulate in
// separate TMEM accumulators (so the small corrections are not added into a
// large running sum).  The tensor core's FP32 accumulation of the leading
// product loses precision with every MMA it adds, and every switch to a fresh
// accumulator costs the tensor pipe about 1.3k idle cycles; the K blocks per
// leading-product accumulator (CB) trade one against the other.  Measured on
// the Rossler workload (4096 trajectories, BF16x6, pointwise error against the
// oracle to t = 5 / far-kernel time): CB = 1 2.7e-8 / 195 ms, CB = 2 1.3e-7 /
// 165 ms, CB = 4 1.8e-6 / 157 ms.  BF16x6 uses CB = 2 (128 rows), three
// buffers rotating while the epilogue warps add each finished one into a
// compensated FP32 pair (TwoSum).  BF16x3 drops products of order 2^-16, far
// above that loss, and keeps CB = 4 (256 rows).  The corrections, 2^-8 of the
// leading term, accumulate in TMEM over the CTA's whole history range and
// are added once.
//
// Warp roles (448 threads): warp 0 TMA producer, warp 1 TMEM owner + MMA
// issuer, warps 2..13 epilogue (lane quarter = warp % 4, 32-column group =
// (warp - 2) / 4).  Fourteen warps put at most four on a sub-partition, so a
// thread may hold 128 registers: the 32 compensated column sums of an
// epilogue thread (64 registers) fit with room for the TMEM staging.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "batched.cuh"
#include "bf16split.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace abm {

namespace {
constexpr int KB = 64;          // history rows per K block (128 bytes of BF16)
constexpr int NCOL = 96;        // columns per tile (32 trajectories x 3)
constexpr int A_BYTES = 128 * KB * 2;
constexpr int B_BYTES = NCOL * KB * 2;
constexpr int EPI_WARPS = 12;   // epilogue warps: 4 lane quarters x 3 column groups
constexpr int ECOLS = NCOL / 3; // columns per epilogue thread
constexpr int THREADS = 32 * (2 + EPI_WARPS);
// Per kind: split products, pieces loaded per operand, ring depths (slots of
// one K block), K blocks per leading-product accumulator.  Shared memory:
// BF16x3 3 x 32 KB Toeplitz + 5 x 24 KB history = 216 KB; BF16x6 2 x 48 KB +
// 3 x 36 KB = 204 KB of the 227 KB a CTA may use.  TMEM (512 columns): three
// 128-column leading-product buffers and one correction accumulator.
template <int KIND> struct FarKind;
template <> struct FarKind<3> {
  static constexpr int NPROD = 3, NP = 2, WST = 3, FST = 5, CB = 4, NBUF = 3;
};
template <> struct FarKind<6> {
  static constexpr int NPROD = 6, NP = 3, WST = 2, FST = 3, CB = 2, NBUF = 3;
};

}  // namespace

// Pre-expanded Toeplitz weights of one alpha: Wx[p][r][x], p = hi/mid/lo.
__global__ void build_wx_kernel(const double* __restrict__ b, const double* __restrict__ a, long long Mw,
                                long long Lbase, long long Lx, __nv_bfloat16* __restrict__ Wx) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // output order
  if (idx >= 128 * Lx) return;
  const int r = (int)((idx >> 6) & 127);
  const long long x = (idx >> 13) * 64 + (idx & 63);
  const long long lag = Lbase - x + (r & 63);
  double w = 0.0;
  if (lag >= 0 && lag <= Mw) w = (r < 64) ? b[lag] : a[lag];
  __nv_bfloat16 pcs[3];
  split3_bf16(w, pcs);
  const size_t plane = (size_t)128 * Lx;
  Wx[idx] = pcs[0];
  Wx[plane + idx] = pcs[1];
  Wx[2 * plane + idx] = pcs[2];
}


template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) far_tc_kernel(FarTcArgs A) {
  using K = FarKind<KIND>;
  constexpr int NA = K::NP, NB = K::NP;  // W and F pieces used
  constexpr int NPROD = K::NPROD;
  // two load rings: Toeplitz blocks (mostly L2 hits, short latency) and
  // history blocks (always from HBM), the second one deeper
  constexpr int WST = K::WST, FST = K::FST;
  constexpr int W_STAGE = NA * A_BYTES, F_STAGE = NB * B_BYTES;
  constexpr int CB = K::CB;      // K blocks per leading-product accumulator
  constexpr int NBUF = K::NBUF;  // leading-product accumulator buffers
  constexpr uint32_t BUF_STRIDE = 128;
  constexpr uint32_t CORR_COL = NBUF * BUF_STRIDE;  // the range-wide correction accumulator
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* smem_f = smem + WST * W_STAGE;
  __shared__ __align__(8) uint64_t wfull[WST], wempty[WST], ffull[FST], fempty[FST], acc_full[NBUF],
      acc_empty[NBUF], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, q = blockIdx.y;
  const int bucket = A.tiles[tile].bucket;
  const int nkb_total = (int)(A.s / KB);
  const int per_q = (nkb_total + A.ksplit - 1) / A.ksplit;
  const int kb_begin = q * per_q;
  int nkb = max(0, min(nkb_total, kb_begin + per_q) - kb_begin);
  if constexpr (kChecked) {
    // every box this CTA loads lies inside its tensor map and every sum it
    // stores inside far; otherwise it loads and stores nothing
    const long long kl = kb_begin + (nkb > 0 ? nkb : 1) - 1;
    const long long yf_last = ((long long)A.tiles[tile].slot * A.f_kblocks + kl) * NCOL + NCOL - 1;
    const long long yw_first = (long long)((A.Lbase - A.s) / KB + kb_begin) * 128;
    const long long yw_last = (long long)((A.Lbase - A.s) / KB + kl) * 128 + 127;
    const long long out_last = (((long long)tile * 2 + 1) * 64 + 63) * NCOL + NCOL - 1;
    if (nkb > 0 && !(in_bounds(A.status, kChkFarTc, yf_last, A.f_map_rows) &&
                     in_bounds(A.status, kChkFarTc, yw_first, A.w_map_rows) &&
                     in_bounds(A.status, kChkFarTc, yw_last, A.w_map_rows) &&
                     in_bounds(A.status, kChkFarTc, out_last, A.far_elems)))
      nkb = 0;
  }
  const int nchunks = (nkb + CB - 1) / CB;
  const int xb0 = (int)((A.Lbase - A.s) / KB);  // Toeplitz block of history block 0

  if (tid == 0) abort_flag = 0;
  if (warp == 1) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int i = 0; i < WST; ++i) { tc::mbar_init(&wfull[i], 1); tc::mbar_init(&wempty[i], 1); }
    for (int i = 0; i < FST; ++i) { tc::mbar_init(&ffull[i], 1); tc::mbar_init(&fempty[i], 1); }
    for (int i = 0; i < NBUF; ++i) { tc::mbar_init(&acc_full[i], 1); tc::mbar_init(&acc_empty[i], EPI_WARPS); }
    tc::mbar_init(&mma_done, 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && nkb > 0) {
      const CUtensorMap* mW = A.tmapW + bucket * 3;
      for (int p = 0; p < NA; ++p) tc::prefetch_tmap(mW + p);
      for (int p = 0; p < NB; ++p) tc::prefetch_tmap(A.tmapF + p);
      // box coordinates of history block kb: Toeplitz block x = Lbase - s + 64 kb, history block (tile, kb)
      auto yw = [&](int kb) { return (xb0 + kb) * 128; };
      const int slot = A.tiles[tile].slot;  // the tile's history pieces
      auto yf = [&](int kb) { return (slot * A.f_kblocks + kb) * NCOL; };
      const uint64_t keep = tc::l2_policy_evict_last(), stream = tc::l2_policy_evict_first();
      // history block j may load once block j - FST has been consumed, Toeplitz
      // block i once block i - WST has: history loads run FST - WST blocks
      // ahead of the Toeplitz loads, issued F(0..lead), then W(i), F(i+lead+1)
      constexpr int lead = FST - WST;
      int nf = 0, nw = 0;  // loads issued per ring
      bool ok = true;
      auto issue_f = [&]() {
        const int fs = nf % FST;
        if (nf >= FST && !tc::mbar_wait(&fempty[fs], ((nf / FST) - 1) & 1, A.budget, &abort_flag)) return false;
        tc::mbar_arrive_expect_tx(&ffull[fs], F_STAGE);
        for (int p = 0; p < NB; ++p)
          tc::tma_load_2d_hint(smem_f + fs * F_STAGE + p * B_BYTES, A.tmapF + p, &ffull[fs], 0,
                               yf(kb_begin + nf), stream);
        ++nf;
        return true;
      };
      for (int j = 0; ok && j <= lead && nf < nkb; ++j) ok = issue_f();
      for (int i = 0; ok && i < nkb; ++i) {
        const int ws = i % WST;
        ok = i < WST || tc::mbar_wait(&wempty[ws], ((i / WST) - 1) & 1, A.budget, &abort_flag);
        if (!ok) break;
        tc::mbar_arrive_expect_tx(&wfull[ws], W_STAGE);
        for (int p = 0; p < NA; ++p)
          tc::tma_load_2d_hint(smem + ws * W_STAGE + p * A_BYTES, mW + p, &wfull[ws], 0, yw(kb_begin + i), keep);
        ++nw;
        if (nf < nkb) ok = issue_f();
      }
      if (!ok) {
        abort_flag = 1;
        report_timeout(A.status, kSiteFarProducer, tile, nw);
        // wait (bounded) for the loads already issued before giving up
        for (int j = max(0, nf - FST); j < nf; ++j) tc::mbar_wait(&ffull[j % FST], (j / FST) & 1, A.budget, nullptr);
        for (int j = max(0, nw - WST); j < nw; ++j) tc::mbar_wait(&wfull[j % WST], (j / WST) & 1, A.budget, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NCOL);
      // (A piece, B piece) of each product: hi=0, mid=1, lo=2
      constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
      constexpr int PB[6] = {0, 1, 0, 2, 1, 0};
      bool first_corr = true;
      int i = 0;  // K block
      for (int c = 0; c < nchunks && !abort_flag; ++c) {
        const int buf = c % NBUF, use = c / NBUF;
        if (use >= 1 && !tc::mbar_wait(&acc_empty[buf], (use - 1) & 1, A.budget, &abort_flag)) {
          abort_flag = 1;
          report_timeout(A.status, kSiteFarAccum, tile, c);
          break;
        }
        tc::fence_after_sync();
        const uint32_t d_main = tmem + buf * BUF_STRIDE;
        const uint32_t d_corr = tmem + CORR_COL;
        bool first_main = true;
        for (const int iend = min(nkb, (c + 1) * CB); i < iend; ++i) {
          const int fs = i % FST, ws = i % WST;
          if (!tc::mbar_wait(&ffull[fs], (i / FST) & 1, A.budget, &abort_flag) ||
              !tc::mbar_wait(&wfull[ws], (i / WST) & 1, A.budget, &abort_flag)) {
            abort_flag = 1;
            report_timeout(A.status, kSiteFarLoad, tile, i);
            break;
          }
          tc::fence_after_sync();
          // descriptors of the two stage bases; every operand is base + a constant
          // offset, added to the 14-bit start-address field (the shared window is
          // below 256 KB, so it cannot carry into the next field)
          const uint64_t ad0 = tc::sdesc_kmajor_sw128(tc::smem_u32(smem + ws * W_STAGE));
          const uint64_t bd0 = tc::sdesc_kmajor_sw128(tc::smem_u32(smem_f + fs * F_STAGE));
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk) {
#pragma unroll
            for (int pr = 0; pr < NPROD; ++pr) {
              const uint64_t ad = ad0 + (uint64_t)((PA[pr] * A_BYTES + kk * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((PB[pr] * B_BYTES + kk * 32) >> 4);
              if (pr == 0) {
                tc::mma_bf16(d_main, ad, bd, idesc, first_main ? 0u : 1u);
                first_main = false;
              } else {
                tc::mma_bf16(d_corr, ad, bd, idesc, first_corr ? 0u : 1u);
                first_corr = false;
              }
            }
          }
          // both slots reusable once these MMAs have read them
          tc::mma_commit(&fempty[fs]);
          tc::mma_commit(&wempty[ws]);
        }
        tc::mma_commit(&acc_full[buf]);  // this chunk's leading-product sum is complete
      }
      // every MMA this thread issued has completed before TMEM is released
      tc::mma_commit(&mma_done);
      tc::mbar_wait(&mma_done, 0, A.budget, nullptr);
    }
  } else {
    // ---------------- epilogue: 12 warps ----------------
    const int lq = warp & 3;           // TMEM lane quarter this warp may access
    const int cg = (warp - 2) >> 2;    // column group: cols 32 cg .. 32 cg + 31
    const uint32_t lane_base = tmem + ((uint32_t)(lq * 32) << 16) + cg * ECOLS;
    constexpr int NG = ECOLS / 16;     // 16-column TMEM loads per accumulator
    // compensated FP32 column sums (hi, lo), two columns per 64-bit register
    // so that the TwoSum runs on packed f32x2 arithmetic (half the instructions)
    uint64_t hi[ECOLS / 2], lo[ECOLS / 2];
#pragma unroll
    for (int j = 0; j < ECOLS / 2; ++j) { hi[j] = 0ull; lo[j] = 0ull; }
    // (hi, lo) += x for the column pair jp, compensated (TwoSum, elementwise)
    auto two_sum2 = [&](int jp, uint64_t x) {
      const uint64_t s = tc::add_f32x2(hi[jp], x);
      const uint64_t bp = tc::sub_f32x2(s, hi[jp]);
      const uint64_t e = tc::add_f32x2(tc::sub_f32x2(hi[jp], tc::sub_f32x2(s, bp)), tc::sub_f32x2(x, bp));
      lo[jp] = tc::add_f32x2(lo[jp], e);
      hi[jp] = s;
    };
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int buf = c % NBUF;
      if (!tc::mbar_wait(&acc_full[buf], (c / NBUF) & 1, A.budget, &abort_flag)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      {
        uint32_t v[NG][16];  // the chunk's leading products: all loads in flight, one wait each
#pragma unroll
        for (int g16 = 0; g16 < NG; ++g16) tc::tmem_ld_32x16_issue(lane_base + buf * BUF_STRIDE + g16 * 16, v[g16]);
#pragma unroll
        for (int g16 = 0; g16 < NG; ++g16) tc::tmem_ld_wait16(v[g16]);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);  // values are in registers
#pragma unroll
        for (int g16 = 0; g16 < NG; ++g16)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            two_sum2(g16 * 8 + j, (uint64_t)v[g16][2 * j] | ((uint64_t)v[g16][2 * j + 1] << 32));
      }
    }
    // the correction products, accumulated over the whole range: into lo
    if (ok && nkb > 0 && tc::mbar_wait(&mma_done, 0, A.budget, &abort_flag)) {
      tc::fence_after_sync();
#pragma unroll
      for (int g16 = 0; g16 < NG; ++g16) {
        uint32_t v[16];
        tc::tmem_ld_32x16_issue(lane_base + CORR_COL + g16 * 16, v);
        tc::tmem_ld_wait16(v);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          lo[g16 * 8 + j] = tc::add_f32x2(lo[g16 * 8 + j], (uint64_t)v[2 * j] | ((uint64_t)v[2 * j + 1] << 32));
      }
    } else {
      ok = false;
    }
    if (ok) {
      // the K-split CTAs of a tile add into one FP64 sum (zeroed before the
      // launch); an unsplit tile stores its sum
      const int r = lq * 32 + lane;    // accumulator row: 0..63 predictor, 64..127 corrector
      const int half = r >> 6, i = r & 63;
      double* out = A.far + (((size_t)tile * 2 + half) * 64 + i) * NCOL + cg * ECOLS;
      auto col = [&](int j) {  // column j's sum: hi + lo of its half of the pair (one FP64 add)
        const int sh = (j & 1) * 32;
        return f32_bits_to_f64((uint32_t)(hi[j >> 1] >> sh)) + f32_bits_to_f64((uint32_t)(lo[j >> 1] >> sh));
      };
      if (A.ksplit == 1) {
#pragma unroll
        for (int j = 0; j < ECOLS; ++j) out[j] = col(j);
      } else {
#pragma unroll
        for (int j = 0; j < ECOLS; ++j) atomicAdd(out + j, col(j));
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}
// Diagnostic path (abm_far_history): split rows [0, s) of a caller's FP64
// history F (rows x 96) into the BF16 planes of column tile 0 (row 0 zero).
__global__ void fill_fsh_kernel(const double* __restrict__ F, long long s, __nv_bfloat16* __restrict__ Fsh,
                                long long plane) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= s * NCOL) return;
  const long long k = idx / NCOL;
  const int col = (int)(idx % NCOL);
  __nv_bfloat16 pcs[3];
  split3_bf16(k == 0 ? 0.0 : F[idx], pcs);
  const size_t o = ((size_t)(k >> 6) * NCOL + col) * 64 + (k & 63);  // K-block tiled, column tile 0
  Fsh[o] = pcs[0];
  Fsh[plane + o] = pcs[1];
  Fsh[2 * plane + o] = pcs[2];
}

// P[i][col] / C[i][col] = sum over the K-split partials of column tile 0.
__global__ void sum_partials_kernel(const double* __restrict__ far, int ksplit, int n_tiles, double* __restrict__ P,
                                    double* __restrict__ C) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * 64 * NCOL) return;
  const int half = idx / (64 * NCOL), rem = idx % (64 * NCOL);
  (half == 0 ? P : C)[rem] = far[(size_t)half * 64 * NCOL + rem];
}

cudaError_t launch_fill_fsh(const double* F, long long s, __nv_bfloat16* Fsh, long long plane, cudaStream_t st) {
  long long n = s * NCOL;
  fill_fsh_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, s, Fsh, plane);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* far, int ksplit, int n_tiles, double* P, double* C, cudaStream_t st) {
  sum_partials_kernel<<<(2 * 64 * NCOL + 255) / 256, 256, 0, st>>>(far, ksplit, n_tiles, P, C);
  return cudaGetLastError();
}

template <int KIND>
size_t far_tc_smem_bytes_t() {
  using K = FarKind<KIND>;
  return (size_t)K::WST * K::NP * A_BYTES + (size_t)K::FST * K::NP * B_BYTES + 1024;
}
size_t far_tc_smem_bytes(int kind) { return kind == 3 ? far_tc_smem_bytes_t<3>() : far_tc_smem_bytes_t<6>(); }

cudaError_t launch_build_wx(const double* b, const double* a, long long Mw, long long Lbase, long long Lx,
                            __nv_bfloat16* Wx, cudaStream_t st) {
  long long n = 128 * Lx;
  build_wx_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, a, Mw, Lbase, Lx, Wx);
  return cudaGetLastError();
}

// static: internal linkage, so the flag below belongs to this build of the
// library (a function-local static of an external template is one object for
// the whole process, shared by every loaded build)
template <int KIND>
static cudaError_t launch_far_tc_t(const FarTcArgs& A, int n_active, cudaStream_t st) {
  const size_t smem = far_tc_smem_bytes_t<KIND>();
  static bool attr = false;  // set once per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(far_tc_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  far_tc_kernel<KIND><<<dim3(n_active, A.ksplit), THREADS, smem, st>>>(A);
  return cudaGetLastError();
}

// kind: 3 = BF16x3, 6 = BF16x6
cudaError_t launch_far_tc(int kind, const FarTcArgs& A, int n_active, cudaStream_t st) {
  if (kind == 3) return launch_far_tc_t<3>(A, n_active, st);
  if (kind == 6) return launch_far_tc_t<6>(A, n_active, st);
  return cudaErrorInvalidValue;
}

// Host: 2D tiled tensor map, BF16, 128-byte swizzle, box {64, box_rows}.
// With inner = 64 it walks a K-block tiled operand as [rows][64].
bool make_tmap_bf16(CUtensorMap* out, void* base, unsigned long long inner, unsigned long long rows,
                    unsigned box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
            cudaSuccess ||
        !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace abm
