// syev3_f64.cu -- FP64 batched 3x3 symmetric eigensolver for sm_103a.
//
// The per-matrix steps of the method of C. F. Borges (arXiv 1806.06698) are
// in solve_f64.cuh; this file holds the kernel that schedules them.
//
// GB300 executes 2 FP64 lanes per SM per clock (1/64 of FP32), so this
// solver is bound by the FP64 pipe, not by HBM.  The kernel is built to spend
// as few FP64 lane-slots per matrix as the method allows:
//  * one matrix per thread; tiles of kTPB packed records arrive by 1-D bulk
//    copy (TMA) into shared memory, double-buffered on two mbarriers, and
//    leave through shared-memory staging with 16-byte stores;
//  * both shifted roots mu and nu are first located in FP32 by the same
//    Borges-Gragg iteration (on the 64x faster pipe), moved right of the root
//    by a bound on the FP32 error, then finished in FP64 by one Borges-Gragg
//    step and the paper's stopping test;
//  * the roots that do not pass (clustered spectra whose root is below FP32
//    resolution, tiny spikes) are compacted with warp ballots into a
//    shared-memory work list and finished by the full FP64 iteration, so that
//    their extra steps occupy ceil(k/32) warps instead of every warp;
//  * reciprocals come from the hardware's 2^-20 estimate and one cubic
//    Newton-Raphson step (<= 1 ulp) instead of IEEE division.

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "serve_tile.cuh"
#include "solve_f64.cuh"

namespace syev3 {
namespace {

using namespace f64;

constexpr int kTPB = 128;        // matrices (threads) per tile
__device__ unsigned g_flags;     // kFlagWaitTimeout when a bulk-copy wait ran out

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------

// kStudy: the method-study build (syev3_batched_method).  The zero finder
// and the deflation test are then chosen at run time by `method`, and
// `counters` receives the 8 method statistics (MethodStat) instead of the
// 4 counters of syev3_batched_ex.  The production build (kStudy = false)
// has these switches compiled out.
// kVectors = false: eigenvalues only (U_out is NULL); the eigenvectors are
// not formed.
// kServe: the serving build.  The tiles are those of the device-resident
// work list `list` (A, n, lam_out and U_out are unused): runs of matrices of
// many requests, each tile with its own input and output rows, solved as one
// ragged batch.  A tile whose input is not 16-byte aligned is loaded with
// plain loads.  The production build (kServe = false) compiles this out.
template <bool kBulkIn, bool kStudy, bool kVectors, bool kServe = false>
__global__ void __launch_bounds__(kTPB) k_syev3_f64(const double* __restrict__ A, int64_t n,
                                                    double* __restrict__ lam_out, double* __restrict__ U_out,
                                                    unsigned long long* __restrict__ counters, Method method,
                                                    const ServeList* __restrict__ list) {
  static_assert(!kServe || (kBulkIn && !kStudy && kVectors), "the serving build is bulk, production, vectors");
  static_assert(kTPB == kServeTile, "serving tiles are solve tiles");
  const int zf = kStudy ? method.zero_finder : kZfProduction;
  const bool eispack = kStudy && method.deflation_test == kDeflEispack;
  __shared__ alignas(16) double s_in[2][kTPB * 6];
  __shared__ alignas(16) double s_lam[kTPB * 3];
  __shared__ alignas(16) double s_U[kTPB * 9];
  // Work list of roots left for the full FP64 iteration: up to two per lane.
  __shared__ double s_hx[2 * kTPB], s_hab[2 * kTPB], s_hb1[2 * kTPB], s_hb2[2 * kTPB], s_hg[2 * kTPB];
  __shared__ bool s_hcap[2 * kTPB];
  __shared__ int s_nhard;
  // Reduced arrows of a pass (struct of arrays W, held in s_U, which is free
  // until the staging writes): slots [0, nc) the arrows carried from the
  // previous pass, then this tile's.  Each pass finishes a whole number of
  // warps' worth of them and carries the rest (< 32) on, so no warp runs the
  // zero finder and the Sec. 1.2 vectors with idle lanes; one last pass
  // after the CTA's final tile finishes the carry.
  constexpr int kW = kTPB + 32;
  static_assert(7 * kW <= 9 * kTPB, "the reduced work list must fit in the staging area");
  double* const s_w = s_U;  // 7 x kW doubles: a1 a2 b1 b2 g c s
  __shared__ int s_we[kW];
  __shared__ int64_t s_wg[kW];  // global index of the matrix
  __shared__ double s_ca[7][32];
  __shared__ int s_ce[32];
  __shared__ int64_t s_cg[32];
  // Rows of this tile's diagonal, deflated and non-finite matrices.
  __shared__ int s_oth[kTPB];
  __shared__ int s_nred, s_noth;
  __shared__ alignas(8) uint64_t s_bar[2];
  // Serving build: the tile of each buffer, and the eigenvector row of each
  // reduced arrow in W and in the carry (s_wg and s_cg then hold the
  // eigenvalue row's address instead of a batch index).
  __shared__ TileRef<double> s_ref[kServe ? 2 : 1];
  __shared__ double* s_wU[kServe ? kW : 1];
  __shared__ double* s_cU[kServe ? 32 : 1];

  const int tid = threadIdx.x, lane_id = tid & 31;
  const unsigned lt_mask = (1u << lane_id) - 1u;
  const int64_t n_tiles = kServe ? list->n_tiles : (n + kTPB - 1) / kTPB;
  bool want_U = (U_out != nullptr);
  bool vec_lam = ((reinterpret_cast<uintptr_t>(lam_out) & 15) == 0);
  bool vec_U = want_U && ((reinterpret_cast<uintptr_t>(U_out) & 15) == 0);
  int64_t cursor = 0;  // serving build: item cursor of the tiles this CTA issues (thread 0)

  if (tid == 0) {
    s_nhard = 0;
    s_nred = 0;
    s_noth = 0;
    if (kBulkIn) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();

  auto issue = [&](int64_t tile, int buf) {
    if constexpr (kServe) {
      const TileRef<double> r = serve_tile<double>(list, tile, cursor);
      s_ref[buf] = r;
      if (reinterpret_cast<uintptr_t>(r.src) & 15) {  // plain loads after the wait
        mbar_arrive(&s_bar[buf]);
        return;
      }
      const uint32_t bytes = (uint32_t)r.cnt * 48u;
      mbar_arrive_expect_tx(&s_bar[buf], bytes);
      bulk_g2s(s_in[buf], r.src, bytes, &s_bar[buf]);
      return;
    }
    const int64_t base = tile * kTPB;
    const int cnt = (int)((n - base) < kTPB ? (n - base) : kTPB);
    const uint32_t bytes = (uint32_t)cnt * 48u;  // 48 = 3 * 16: always a multiple of 16
    mbar_arrive_expect_tx(&s_bar[buf], bytes);
    bulk_g2s(s_in[buf], A + base * 6, bytes, &s_bar[buf]);
  };

  auto lane_of_record = [&](const double* rec) {
    const double2* src = reinterpret_cast<const double2*>(rec);
    const double2 p0 = src[0], p1 = src[1], p2 = src[2];
    const double a[6] = {p0.x, p0.y, p1.x, p1.y, p2.x, p2.y};
    return eispack ? make_lane<true>(a) : make_lane<false>(a);
  };

  uint32_t phases = 0u;  // bit b: parity of the next completion of s_bar[b]
  int buf = 0;
  int nc = 0;            // reduced arrows carried into this pass (CTA-uniform)
  int64_t tile = blockIdx.x;
  if (kBulkIn && tid == 0 && tile < n_tiles) issue(tile, 0);

  for (;; tile += gridDim.x, buf ^= 1) {
    const bool flush = (tile >= n_tiles);  // the pass that finishes the carry
    if (flush && nc == 0) break;
    const int64_t base = tile * kTPB;
    int cnt = flush ? 0 : (int)((n - base) < kTPB ? (n - base) : kTPB);
    const int64_t next = tile + gridDim.x;
    if (!flush) {
      if (kBulkIn) {
        if (tid == 0 && next < n_tiles) issue(next, buf ^ 1);
        const bool ok = mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
        if (__syncthreads_or(!ok)) {
          // Lost wait (CTA-uniform decision): flag it, give the copies in
          // flight a second bounded chance to land so that no write into
          // shared memory outlives the CTA, and stop.
          if (tid == 0) atomicOr(&g_flags, kFlagWaitTimeout);
          mbar_wait(&s_bar[buf], (phases >> buf) & 1u);
          if (next < n_tiles) mbar_wait(&s_bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
          return;
        }
        phases ^= 1u << buf;
        if constexpr (kServe) {
          const TileRef<double> r = s_ref[buf];
          cnt = r.cnt;
          want_U = (r.U != nullptr);
          vec_lam = ((reinterpret_cast<uintptr_t>(r.lam) & 15) == 0);
          vec_U = want_U && ((reinterpret_cast<uintptr_t>(r.U) & 15) == 0);
          if (reinterpret_cast<uintptr_t>(r.src) & 15) {
            for (int i = tid; i < cnt * 6; i += kTPB) s_in[buf][i] = r.src[i];
            __syncthreads();
          }
        }
      } else {
        for (int i = tid; i < cnt * 6; i += kTPB) s_in[buf][i] = A[base * 6 + i];
        __syncthreads();
      }
    }

    // Phase A: the carried arrows take W's first slots; each thread reduces
    // its own matrix to an arrow and classifies it; reduced arrows are
    // appended to W, the rows of the other classes listed for phase E.
    if (tid < nc) {
#pragma unroll
      for (int f = 0; f < 7; ++f) s_w[f * kW + tid] = s_ca[f][tid];
      s_we[tid] = s_ce[tid];
      s_wg[tid] = s_cg[tid];
      if constexpr (kServe) s_wU[tid] = s_cU[tid];
    }
    {
      Lane A0;
      A0.cls = kIdle;
      if (tid < cnt) A0 = lane_of_record(&s_in[buf][tid * 6]);
      const bool red = (A0.cls == kReduced);
      const bool oth = (A0.cls != kReduced) && (A0.cls != kIdle);
      const unsigned mr = __ballot_sync(0xffffffffu, red);
      const unsigned mo = __ballot_sync(0xffffffffu, oth);
      int rb = 0, ob = 0;
      if (lane_id == 0) {
        if (mr) rb = atomicAdd(&s_nred, __popc(mr));
        if (mo) ob = atomicAdd(&s_noth, __popc(mo));
      }
      rb = __shfl_sync(0xffffffffu, rb, 0);
      ob = __shfl_sync(0xffffffffu, ob, 0);
      if (red) {
        const int slot = nc + rb + __popc(mr & lt_mask);
        s_w[0 * kW + slot] = A0.a1;
        s_w[1 * kW + slot] = A0.a2;
        s_w[2 * kW + slot] = A0.b1;
        s_w[3 * kW + slot] = A0.b2;
        s_w[4 * kW + slot] = A0.g;
        s_w[5 * kW + slot] = A0.c;
        s_w[6 * kW + slot] = A0.s;
        s_we[slot] = A0.e;
        if constexpr (kServe) {
          const TileRef<double> r = s_ref[buf];
          s_wg[slot] = (int64_t)reinterpret_cast<uintptr_t>(r.lam + tid * 3);
          s_wU[slot] = r.U ? r.U + tid * 9 : nullptr;
        } else {
          s_wg[slot] = base + tid;
        }
      }
      if (oth) s_oth[ob + __popc(mo & lt_mask)] = tid;
      if (kStudy && counters != nullptr) {
        const unsigned md = __ballot_sync(0xffffffffu, A0.cls == kDiagonal);
        const unsigned mf = __ballot_sync(0xffffffffu, A0.cls == kDeflated);
        if (lane_id == 0) {
          if (md) atomicAdd(&counters[kStatDiagonal], (unsigned long long)__popc(md));
          if (mf) atomicAdd(&counters[kStatDeflated], (unsigned long long)__popc(mf));
          if (mr) atomicAdd(&counters[kStatReduced], (unsigned long long)__popc(mr));
        }
      }
    }
    __syncthreads();
    const int n_avail = nc + s_nred, n_oth = s_noth;
    // This pass finishes P arrows: whole warps (all of them in the last pass).
    const int P = flush ? n_avail : min(kTPB, n_avail & ~31);
    const int nc_next = n_avail - P;
    if (tid < nc_next) {
#pragma unroll
      for (int f = 0; f < 7; ++f) s_ca[f][tid] = s_w[f * kW + P + tid];
      s_ce[tid] = s_we[P + tid];
      s_cg[tid] = s_wg[P + tid];
      if constexpr (kServe) s_cU[tid] = s_wU[P + tid];
    }
    Lane L;
    L.cls = kIdle;
    int64_t gidx = -1;
    double* urow = nullptr;  // serving build: the arrow's eigenvector row (null: none wanted)
    if (tid < P) {
      L.a1 = s_w[0 * kW + tid];
      L.a2 = s_w[1 * kW + tid];
      L.b1 = s_w[2 * kW + tid];
      L.b2 = s_w[3 * kW + tid];
      L.g = s_w[4 * kW + tid];
      L.c = s_w[5 * kW + tid];
      L.s = s_w[6 * kW + tid];
      L.e = s_we[tid];
      L.cls = kReduced;
      gidx = s_wg[tid];
      if constexpr (kServe) urow = s_wU[tid];
    }

    // Phases B, C: FP32 seeds, then one FP64 step and the stopping test.
    // Problem 0 is mu (A - a1 I), problem 1 is nu (P(a2 I - A)P: spikes
    // swapped), Sec. 1.2.
    const bool reduced = (L.cls == kReduced);
    double root[2] = {0.0, 0.0};
    bool hard[2] = {false, false};
    double ab = 0.0, pb1[2] = {0.0, 0.0}, pb2[2] = {0.0, 0.0}, pg[2] = {0.0, 0.0};
    if (reduced && zf != kZfProduction) {
      // Study: every root goes to the full FP64 iteration from the paper's
      // own start (Eq. (7) for Borges-Gragg, Sec. 1.4.2 for Newton).
      ab = L.a1 - L.a2;
      pb1[0] = L.b1 * L.b1; pb2[0] = L.b2 * L.b2; pg[0] = L.g - L.a1;
      pb1[1] = pb2[0]; pb2[1] = pb1[0]; pg[1] = L.a2 - L.g;
      hard[0] = hard[1] = true;
    } else if (reduced) {
      ab = L.a1 - L.a2;
      const double bb1 = L.b1 * L.b1, bb2 = L.b2 * L.b2;
      pb1[0] = bb1; pb2[0] = bb2; pg[0] = L.g - L.a1;
      pb1[1] = bb2; pb2[1] = bb1; pg[1] = L.a2 - L.g;
      // FP32 can carry the problem when its data are normal FP32 numbers
      // with room for the products formed from them: spikes^2 >= 2^-120
      // (a tiny spike gives a root near its own size, 1/x^2 terms up to
      // ~2^120) and abar >= 2^-100.  An FP32 value that still underflows only
      // makes the FP64 step more cautious or sends the root to the full
      // iteration; acceptance is always the FP64 stopping test.
      const bool fp32_ok = hi_mag(bb1) >= hi_pow2(-120) && hi_mag(bb2) >= hi_pow2(-120) &&
                           hi_mag(ab) >= hi_pow2(-100);  // (all three >= 0)
      float sd[2] = {0.f, 0.f};
      double pc[2] = {0.0, 0.0}, pK[2] = {0.0, 0.0};
      const float fab = d2f_rn(ab), fb1[2] = {d2f_rn(pb1[0]), d2f_rn(pb1[1])}, fb2[2] = {d2f_rn(pb2[0]), d2f_rn(pb2[1])};
      if (fp32_ok) {
        const double rab = rcp64(ab);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          pc[k] = pb2[k] * rab;
          pK[k] = -pg[k] - pc[k];
        }
        const float fg[2] = {d2f_rn(pg[0]), d2f_rn(pg[1])};
        const float fc[2] = {d2f_rn(pc[0]), d2f_rn(pc[1])}, fK[2] = {d2f_rn(pK[0]), d2f_rn(pK[1])};
        seed32x2(fab, fb1, fb2, fg, fc, fK, sd);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        double x = f2d_exact(sd[k]);
        int st = 2;
        // 2^-900 <= x <= 2^100 (x >= 0): the range finish64 assumes.
        if (hi_mag(x) >= hi_pow2(-900) && dbits(x) <= dbits(0x1p+100))
          st = finish64(ab, pb1[k], pb2[k], pg[k], pc[k], pK[k], fab, fb1[k], fb2[k], x);
        root[k] = (st == 2) ? 0.0 : x;  // 0: restart from Eq. (7)
        hard[k] = (st != 0);
      }
    }

    // Phase D: compact the unfinished roots into the shared work list and
    // finish them with every lane of the CTA available.  (Its first barrier
    // also orders every read of W above before the staging writes below.)
    int slot[2] = {-1, -1};
    {
      const unsigned m0 = __ballot_sync(0xffffffffu, hard[0]);
      const unsigned m1 = __ballot_sync(0xffffffffu, hard[1]);
      const int total = __popc(m0) + __popc(m1);
      int wbase = 0;
      if (lane_id == 0 && total) wbase = atomicAdd(&s_nhard, total);
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (hard[0]) slot[0] = wbase + __popc(m0 & lt_mask);
      if (hard[1]) slot[1] = wbase + __popc(m0) + __popc(m1 & lt_mask);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (slot[k] >= 0) {
          s_hx[slot[k]] = root[k];
          s_hab[slot[k]] = ab;
          s_hb1[slot[k]] = pb1[k];
          s_hb2[slot[k]] = pb2[k];
          s_hg[slot[k]] = pg[k];
        }
      }
    }
    __syncthreads();
    const int n_hard = s_nhard;
    for (int i = tid; i < n_hard; i += kTPB) {
      bool cp;
      int steps;
      if (zf == kZfNewton)
        s_hx[i] = zero_newton_full(s_hab[i], s_hb1[i], s_hb2[i], s_hg[i], cp, steps);
      else
        s_hx[i] = zero_bg_full(s_hab[i], s_hb1[i], s_hb2[i], s_hg[i], s_hx[i], cp, steps);
      s_hcap[i] = cp;
      if (kStudy && counters != nullptr) {
        // Steps, and the lane-slots the warp spent on them: on the FP64 pipe
        // an instruction occupies all 32 lanes, so a warp costs 32 x its
        // longest iteration.
        const unsigned am = __activemask();
        const unsigned sum = __reduce_add_sync(am, (unsigned)steps);
        const unsigned mx = __reduce_max_sync(am, (unsigned)steps);
        if ((tid & 31) == __ffs(am) - 1) {
          atomicAdd(&counters[kStatSteps], (unsigned long long)sum);
          atomicAdd(&counters[kStatRoots], (unsigned long long)__popc(am));
          atomicAdd(&counters[kStatWarpSlots], 32ull * mx);
        }
      }
    }
    __syncthreads();
    bool capped = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (slot[k] >= 0) {
        root[k] = s_hx[slot[k]];
        capped |= s_hcap[slot[k]];
      }
    }

    // Phase E: eigenpairs of the reduced arrow of slot tid (staged when it
    // belongs to this tile, written straight to memory when carried in), then
    // of one of this tile's other matrices (re-reduced from its record, which
    // is still in shared memory).
    if (reduced && !kVectors) {
      double lam[3];
      finish_values(L, root[0], root[1], lam);
      const int64_t row = gidx - base;
      if (row >= 0 && row < cnt) {
#pragma unroll
        for (int k = 0; k < 3; ++k) s_lam[row * 3 + k] = lam[k];
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) lam_out[gidx * 3 + k] = lam[k];
      }
    } else if (reduced) {
      double lam[3], U[9];
      finish_lane(L, root[0], root[1], lam, U);
      int64_t row;
      if constexpr (kServe) {
        // Byte offset of the arrow's eigenvalue row from this tile's first row.
        const int64_t d = flush ? -1
                                : (int64_t)(uintptr_t)gidx - (int64_t)reinterpret_cast<uintptr_t>(s_ref[buf].lam);
        row = (d >= 0 && d < (int64_t)cnt * 24) ? d / 24 : -1;
      } else {
        row = gidx - base;
      }
      if (row >= 0 && row < cnt) {
#pragma unroll
        for (int k = 0; k < 3; ++k) s_lam[row * 3 + k] = lam[k];
#pragma unroll
        for (int k = 0; k < 9; ++k) s_U[row * 9 + k] = U[k];
      } else if constexpr (kServe) {
        double* lrow = reinterpret_cast<double*>((uintptr_t)gidx);
#pragma unroll
        for (int k = 0; k < 3; ++k) lrow[k] = lam[k];
        if (urow != nullptr) {
#pragma unroll
          for (int k = 0; k < 9; ++k) urow[k] = U[k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) lam_out[gidx * 3 + k] = lam[k];
        if (want_U) {
#pragma unroll
          for (int k = 0; k < 9; ++k) U_out[gidx * 9 + k] = U[k];
        }
      }
    }
    bool nonfinite = false;
    if (tid < n_oth) {
      const int row = s_oth[tid];
      const Lane O = lane_of_record(&s_in[buf][row * 6]);
      double lam[3], U[9];
      if (O.cls == kNonFinite) {
        nonfinite = true;
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
        for (int k = 0; k < 3; ++k) lam[k] = qnan;
#pragma unroll
        for (int k = 0; k < 9; ++k) U[k] = qnan;
      } else if (kVectors) {
        finish_lane(O, 0.0, 0.0, lam, U);
      } else {
        finish_values(O, 0.0, 0.0, lam);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) s_lam[row * 3 + k] = lam[k];
      if (kVectors) {
#pragma unroll
        for (int k = 0; k < 9; ++k) s_U[row * 9 + k] = U[k];
      }
    }
    if (counters != nullptr) {
      const unsigned cm = __ballot_sync(0xffffffffu, capped);
      const unsigned nf = __ballot_sync(0xffffffffu, nonfinite);
      if (lane_id == 0) {
        if (cm) atomicAdd(&counters[0], (unsigned long long)__popc(cm));
        if (nf) atomicAdd(&counters[1], (unsigned long long)__popc(nf));
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_nhard = 0;
      s_nred = 0;
      s_noth = 0;
    }

    // Coalesced write-back of the tile: 16-byte stores where aligned.  The
    // rows of arrows carried to the next pass receive their results then.
    if (!flush) {
      double* dst = kServe ? s_ref[buf].lam : lam_out + base * 3;
      const int m = cnt * 3;
      if (vec_lam) {
        double2* d2 = reinterpret_cast<double2*>(dst);
        const double2* s2 = reinterpret_cast<const double2*>(s_lam);
        for (int i = tid; i < m / 2; i += kTPB) d2[i] = s2[i];
        if ((m & 1) && tid == 0) dst[m - 1] = s_lam[m - 1];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_lam[i];
      }
    }
    if (!flush && want_U) {
      double* dst = kServe ? s_ref[buf].U : U_out + base * 9;
      const int m = cnt * 9;
      if (vec_U) {
        double2* d2 = reinterpret_cast<double2*>(dst);
        const double2* s2 = reinterpret_cast<const double2*>(s_U);
        for (int i = tid; i < m / 2; i += kTPB) d2[i] = s2[i];
        if ((m & 1) && tid == 0) dst[m - 1] = s_U[m - 1];
      } else {
        for (int i = tid; i < m; i += kTPB) dst[i] = s_U[i];
      }
    }
    __syncthreads();
    nc = nc_next;
    if (flush) break;
  }
}

template <bool kBulkIn, bool kStudy, bool kVectors, bool kServe = false>
int blocks_per_sm_f64() {
  static int cached = -1;
  if (cached < 0) {
    int v = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &v, k_syev3_f64<kBulkIn, kStudy, kVectors, kServe>, kTPB, 0);
    cached = (e == cudaSuccess && v > 0) ? v : 1;
  }
  return cached;
}

template <bool kBulkIn, bool kStudy, bool kVectors = true>
cudaError_t launch_f64_t(const double* A, int64_t n, double* lam, double* U, unsigned long long* counters,
                         Method method, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (n + kTPB - 1) / kTPB;
  const int64_t resident = (int64_t)sms * blocks_per_sm_f64<kBulkIn, kStudy, kVectors>();
  const int grid = (int)(n_tiles < resident ? n_tiles : resident);
  k_syev3_f64<kBulkIn, kStudy, kVectors><<<grid, kTPB, 0, stream>>>(A, n, lam, U, counters, method, nullptr);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_f64_serve(const ServeList* list, unsigned long long* counters, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // The list's length is known only on the device: a resident grid; CTAs
  // without a tile exit at once.
  const int grid = sms * blocks_per_sm_f64<true, false, true, true>();
  const Method m{kZfProduction, kDeflSimplified};
  k_syev3_f64<true, false, true, true><<<grid, kTPB, 0, stream>>>(nullptr, 0, nullptr, nullptr, counters, m, list);
  return cudaGetLastError();
}

cudaError_t launch_f64(const double* A, int64_t n, double* lam, double* U, unsigned long long* counters,
                       cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const Method m{kZfProduction, kDeflSimplified};
  if ((reinterpret_cast<uintptr_t>(A) & 15) == 0) {
    if (U == nullptr) return launch_f64_t<true, false, false>(A, n, lam, U, counters, m, stream);
    return launch_f64_t<true, false>(A, n, lam, U, counters, m, stream);
  }
  return launch_f64_t<false, false>(A, n, lam, U, counters, m, stream);
}

cudaError_t launch_f64_method(const double* A, int64_t n, double* lam, double* U, unsigned long long* stats,
                              Method method, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(A) & 15) == 0)
    return launch_f64_t<true, true>(A, n, lam, U, stats, method, stream);
  return launch_f64_t<false, true>(A, n, lam, U, stats, method, stream);
}

// The failure path of the bounded waits, exercised: one thread waits on an
// mbarrier that nothing completes (no copy is issued, nothing arrives), so
// the wait runs out after kWaitLimitNs and the timeout bit is recorded, as a
// lost bulk copy would record it.
__global__ void k_wait_selftest() {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if (!mbar_wait(&bar, 0)) atomicOr(&g_flags, kFlagWaitTimeout);
  }
}

cudaError_t launch_wait_selftest(cudaStream_t stream) {
  k_wait_selftest<<<1, 32, 0, stream>>>();
  return cudaGetLastError();
}

cudaError_t take_flags_f64(unsigned* flags) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_flags, sizeof(v));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_flags, &zero, sizeof(zero));
  *flags |= v;
  return e;
}

}  // namespace syev3
