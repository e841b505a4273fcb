// Lasso path by cyclic coordinate descent with GAP SAFE sphere screening
// (Fercoq, Gramfort, Salmon, ICML 2015, Algorithm 1) as one persistent
// cooperative kernel on a GB300.
//
// One lambda of the grid (Sec. 3.3 warm start, Sec. 4.1 schedule):
//   check   (all CTAs)  c~ = X^T rho in FP32 with a forward-error bound per
//                       feature; exact double-float recomputation of the
//                       features the bound leaves undecided (the maximum used
//                       by the dual point, Eq. (8), and the sphere test,
//                       Eq. (7) with the radius of Eq. (10)); FP64 objectives,
//                       gap and radius (Prop. 1); compaction of the
//                       safe-active set (Eq. (6)).
//   f passes            each pass over the safe-active list runs in rounds:
//     chain   (CTA 0)   the coordinates whose coefficient is nonzero, in
//                       ascending order, one after the other; columns are
//                       staged by bulk copies into a shared-memory ring, the
//                       residual lives in registers, and the residual after
//                       every step is kept as a snapshot.
//     verify  (all)     every other coordinate of the pass has a zero
//                       coefficient; it stays zero iff |x_j^T rho| <= lambda
//                       for the residual in force at its position (the
//                       snapshot of its segment).  All of them are tested at
//                       once; the first one that would move ends the round:
//                       the chain is rolled back to that position, the round
//                       after it starts with that coordinate.
//   A zero coefficient that stays zero leaves rho unchanged, so the iterates
//   are those of plain cyclic coordinate descent over the safe-active set.
//
// Options of the check: the GAP SAFE dome of Eq. (11) beside the sphere, and
// the sphere radius of Thm. 2.  Instantiations with EN = true solve the
// Elastic-Net of the paper's appendix as the Lasso on the augmented design
// [X; sqrt(mu) I], whose extra rows stay implicit.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "cd_common.cuh"
#include "internal.h"

namespace lassogs {

// certificate values of a position: a chain entry (never verified), or a zero
// coefficient without a valid certificate (always verified)
constexpr float kSkChain = 3.0e38f;
constexpr float kSkNone = -3.0e38f;

struct Ctrl {
  unsigned bar_count, bar_gen;
  int err;
  int nonfinite;
  double lambda_max, yy, eps;
  unsigned long long m_bits;  // max |x_j^T rho| over the scope (exact), ordered bits
  unsigned mlo_bits;          // max (|c~_j| - E_j), FP32 bits
  int fstar;                  // first entering position of a round
  int nzl;                    // zero-list length (coefficients removed by screening)
  int q, s;                   // safe-active and support counts
  int pos, round_end, nc, done, sup_idx, forced, n_entered;
  float rho_bound;            // bound on ||rho|| for every snapshot of a round
  int failed;                 // lockstep batches: error code of a problem that failed earlier
  float mcur;                 // movement bound: sum |delta_c| ||x_c|| since the last check (rounded up)
  // cycle counters of CTA 0 by phase (check, chain, verify, rollback/accept,
  // end of pass, setup of a round) and event counts (rounds, rollbacks)
  unsigned long long prof[8];
  int win;                    // positions a round may span (adaptive, see the passes)
  int prob;                   // groups of CTAs: the problem CTA 0 took from the queue
};

struct Args {
  const float* Xh;  // n x p column-major FP32 (or the high plane of an FP64 X)
  const float* Xl;  // low plane of an FP64 X, or nullptr
  long long ldx;    // column stride of Xh / Xl (a multiple of 4)
  long long ldw;    // leading dimension of the residual planes and snapshots (4 * ld4)
  int n, p, ld4;    // ld4 = ceil(n / 4) float4 granules per column
  int T, words;
  int fs;           // features per CTA slice (multiple of 32)
  int s_cap;        // max chain entries per round
  int f;            // screen period
  int dual_point, xtr_scope, warm_start;
  int screen_rule;  // 0: GAP SAFE sphere; 1: sphere and GAP SAFE dome
  int refined_radius;  // 1: the sphere radius of Thm. 2
  double enet_alpha;   // Elastic-Net mixing a (1 = the Lasso)
  long long max_epochs;
  const double* y;
  const double* ratios;
  double* beta_out;
  uint32_t* mask_out;
  lasso_path_stats* stats;
  // workspace: CTA c uses ws + c * cta_bytes (cta_bytes = 0: one shared copy)
  char* ws;
  size_t cta_bytes;
  size_t o_ctrl, o_cnt_kept, o_cnt_sup, o_cnt_nnz, o_cnt_zero, o_part_l1, o_nrm, o_nrmf, o_ftab, o_bdf, o_b0df,
      o_rho_h, o_rho_l, o_rho0_h, o_rho0_l, o_ctil, o_mask, o_A, o_sup0, o_sup1, o_chain, o_entered, o_oldb, o_recs,
      o_snap, o_zl_j, o_zl_b, o_zbits, o_yb, o_sk, o_mref, o_msnap, o_cy, o_part_l2;
  // batched solver: B problems over the same X, problem b uses column b of Y
  // (ld ldy) and the rows i with rmask[i + b * ldm] != 0 (all rows if null)
  int B;
  long long ldy, ldm;
  const uint8_t* rmask;
  const double* beta0;  // starting points beta0[j + b * ldb0], or null
  long long ldb0;
  int* queue;       // next problem to take
  int gsize;        // CTAs per problem (a group shares one workspace region and its barrier)
  double tol;       // gap_tol_rel
  // lockstep batches: one launch per lambda range [t0, t1), workspace region
  // per problem (not per CTA), and the first check of each lambda reads
  // cfirst[j + b * ldc] with the forward-error factor cfactor
  int lockstep, t0, t1;
  const float* cfirst;
  long long ldc;
  float cfactor;
};

// Fields the shared helpers read (see cd_common.cuh), built from a CTA's
// workspace base.
struct ChainCtx {
  const float* Xh;
  const float* Xl;
  long long ldx, ldw;
  int n, ld4;
  const int* A;
  const int* chain;
  const float4* ftab;
  float2* bdf;
  const float* nrmf;
  ChainRec* recs;
  float2* oldb;
  float* snap;
  float* msnap;
};

__device__ __forceinline__ int slice_begin(const Args& a, int c) {
  long long v = (long long)c * a.fs;
  return v < a.p ? (int)v : a.p;
}

// Row bits of the chain thread's granules for problem b: bit 4k + c is set
// when row 4 (tid + 128 k) + c belongs to the problem's row subset.
template <int NGC, int CW>
__device__ __forceinline__ uint32_t chain_row_bits(const Args& a, int b) {
  const int tid = threadIdx.x;
  uint32_t bits = 0;
#pragma unroll
  for (int k = 0; k < NGC; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int row = 4 * (tid + 32 * CW * k) + c;
      const bool in = row < a.n && (a.rmask == nullptr || a.rmask[row + (size_t)b * a.ldm] != 0);
      bits |= (in ? 1u : 0u) << (4 * k + c);
    }
  return bits;
}

// rows of a batched problem's residual held by one thread while beta0 is applied
constexpr int kBatchRowsPerThread = 8;
static_assert(kBatchRowsPerThread * kThreads >= kMaxRows, "a thread's rows must cover n <= kMaxRows");

// Support function of the dome D(c, rad, al, nrm) at a vector x, from c^T x,
// nrm^T x and ||x|| (the paper's appendix, dome test).  The dome is the part
// of the ball B(c, rad) with nrm^T (z - c) <= -al rad.  When x points far
// enough against nrm the ball's extreme point c + rad x/||x|| lies in the
// dome; otherwise the maximum is on the circle where the hyperplane cuts the
// sphere.
__device__ __forceinline__ double dome_support(double xc, double rad, double al, double xnr, double xn) {
  if (xnr < __dmul_rn(-al, xn)) return __dadd_rn(xc, __dmul_rn(rad, xn));
  double w = __dsub_rn(__dmul_rn(xn, xn), __dmul_rn(xnr, xnr));
  if (w < 0.0) w = 0.0;
  return __dadd_rn(__dsub_rn(xc, __dmul_rn(__dmul_rn(rad, al), xnr)),
                   __dmul_rn(rad, __dsqrt_rn(__dmul_rn(w, __dsub_rn(1.0, __dmul_rn(al, al))))));
}

// Per-problem set-up of a batched problem (the single path does this with the
// precompute kernels): y restricted to the problem's rows, rho = y - X beta0,
// ||y||^2, and for every column the norm over those rows and x_j^T y, whose
// largest magnitude is lambda_max (Sec. 1.2).  FP64 accumulation.  The parts:
// reset (the control fields a problem starts from), rows (y, rho, ||y||^2),
// the columns [j0, j1) and final (lambda_max and the input checks).  One CTA
// per problem runs them all; in a group of CTAs every CTA runs the columns of
// its slice, CTA 0 the rest, with group barriers in between.
template <bool XLO>
__device__ void batch_setup(const Args& a, Ctrl* ctl, char* wsb, int b, double* dbuf, int j0, int j1, bool reset,
                            bool rows, bool final) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kThreads / 32;
  double* yb = reinterpret_cast<double*>(wsb + a.o_yb);
  float* rh = reinterpret_cast<float*>(wsb + a.o_rho_h);
  float* rl = reinterpret_cast<float*>(wsb + a.o_rho_l);
  float* r0h = reinterpret_cast<float*>(wsb + a.o_rho0_h);
  float* r0l = reinterpret_cast<float*>(wsb + a.o_rho0_l);
  double* nrm = reinterpret_cast<double*>(wsb + a.o_nrm);
  float* nrmf = reinterpret_cast<float*>(wsb + a.o_nrmf);
  float4* ftab = reinterpret_cast<float4*>(wsb + a.o_ftab);
  float2* bdf = reinterpret_cast<float2*>(wsb + a.o_bdf);
  float2* b0df = reinterpret_cast<float2*>(wsb + a.o_b0df);
  double* cy = reinterpret_cast<double*>(wsb + a.o_cy);
  if (reset) {
    if (tid == 0) {
      ctl->err = 0;
      ctl->nonfinite = 0;
      ctl->m_bits = 0ull;
      ctl->mlo_bits = 0u;
      ctl->nzl = 0;
    }
    __syncthreads();
  }
  double yy = 0.0;
  bool finite = true;
  for (int i = tid; rows && i < a.ldw; i += kThreads) {
    const bool in = i < a.n && (a.rmask == nullptr || a.rmask[i + (size_t)b * a.ldm] != 0);
    const double v = in ? a.y[i + (size_t)b * a.ldy] : 0.0;
    finite = finite && isfinite(v);
    yb[i] = v;
    yy = __fma_rn(v, v, yy);
    const df2 d = df_from_double(v);
    rh[i] = d.h;
    rl[i] = d.l;
    r0h[i] = d.h;
    r0l[i] = d.l;
  }
  if (rows) {
    yy = block_sum_d(yy, dbuf);
    if (tid == 0) ctl->yy = yy;
  }
  for (int j = j0 + warp; j < j1; j += nwarps) {
    const float* col = a.Xh + (long long)j * a.ldx;
    const float* coll = XLO ? a.Xl + (long long)j * a.ldx : nullptr;
    double s2 = 0.0, sy = 0.0;
    bool fin = true;
    for (int i = lane; i < a.n; i += 32) {
      const bool in = a.rmask == nullptr || a.rmask[i + (size_t)b * a.ldm] != 0;
      double x = in ? (double)__ldg(col + i) : 0.0;
      if (XLO && in) x = __dadd_rn(x, (double)__ldg(coll + i));
      fin = fin && isfinite(x);
      s2 = __fma_rn(x, x, s2);
      sy = __fma_rn(x, in ? a.y[i + (size_t)b * a.ldy] : 0.0, sy);
    }
    s2 = warp_sum_d(s2);
    sy = warp_sum_d(sy);
    fin = __all_sync(0xffffffffu, fin);
    if (lane == 0) {
      if (!fin || !isfinite(sy)) finite = false;
      const double nr = __dsqrt_rn(s2);
      nrm[j] = nr;
      nrmf[j] = __double2float_ru(nr);
      cy[j] = sy;
      const df2 iv = df_from_double(s2 > 0.0 ? __drcp_rn(s2) : 0.0);
      ftab[j] = make_float4(iv.h, iv.l, 0.f, 0.f);
      if (isfinite(sy)) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(fabs(sy)));
      const df2 bd = df_from_double(a.beta0 ? a.beta0[j + (size_t)b * a.ldb0] : 0.0);
      bdf[j] = make_float2(bd.h, bd.l);
      b0df[j] = make_float2(bd.h, bd.l);
    }
  }
  if (rows && a.beta0 != nullptr) {
    // rho = y - X beta0 on the problem's rows: the nonzero terms are
    // subtracted in ascending j, each product and difference rounded once
    __shared__ int s_j[kThreads];
    __shared__ double s_b[kThreads];
    __shared__ int s_cnt[kThreads / 32];
    double racc[kBatchRowsPerThread];
    unsigned inrow = 0;
#pragma unroll
    for (int k = 0; k < kBatchRowsPerThread; ++k) {
      const int i = tid + k * kThreads;
      const bool in = i < a.n && (a.rmask == nullptr || a.rmask[i + (size_t)b * a.ldm] != 0);
      inrow |= (in ? 1u : 0u) << k;
      racc[k] = in ? yb[i] : 0.0;
    }
    const double* b0 = a.beta0 + (size_t)b * a.ldb0;
    for (int base = 0; base < a.p; base += kThreads) {
      const int j = base + tid;
      const double v = j < a.p ? b0[j] : 0.0;
      finite = finite && isfinite(v);
      int tot;
      const int r = block_rank(v != 0.0, s_cnt, &tot);
      if (v != 0.0) {
        s_j[r] = j;
        s_b[r] = v;
      }
      __syncthreads();
      for (int c = 0; c < tot; ++c) {
        const long long off = (long long)s_j[c] * a.ldx;
        const double bv = s_b[c];
#pragma unroll
        for (int k = 0; k < kBatchRowsPerThread; ++k) {
          if ((inrow >> k) & 1u) {
            const int i = tid + k * kThreads;
            double x = (double)a.Xh[off + i];
            if (XLO) x = __dadd_rn(x, (double)a.Xl[off + i]);
            racc[k] = __dsub_rn(racc[k], __dmul_rn(bv, x));
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kBatchRowsPerThread; ++k) {
      const int i = tid + k * kThreads;
      if ((inrow >> k) & 1u) {
        finite = finite && isfinite(racc[k]);
        const df2 d = df_from_double(racc[k]);
        rh[i] = d.h;
        rl[i] = d.l;
        r0h[i] = d.h;
        r0l[i] = d.l;
      }
    }
  }
  if (!finite) atomicExch(&ctl->nonfinite, 1);
  __syncthreads();
  if (final) {
    if (tid == 0) {
      ctl->lambda_max = __longlong_as_double((long long)ctl->m_bits);
      ctl->m_bits = 0ull;
      ctl->eps = a.tol * ctl->yy;
      bool bad = !(ctl->lambda_max > 0.0);
      for (int t = 0; t < a.T; ++t) bad = bad || !(a.ratios[t] > 0.0 && a.ratios[t] <= 1.0);
      if (ctl->nonfinite) ctl->err = kErrNonfinite;
      else if (bad) ctl->err = kErrInvalidArg;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- the kernel
// BATCH = false: the whole grid cooperates on one problem (grid barriers).
// BATCH = true: groups of a.gsize CTAs (one CTA by default) each have their
// own workspace region, whose control block carries the group's barrier, and
// solve problems taken from a queue, one whole path at a time; within a group
// the CTAs split the features into slices as the single path does.
// MINB: CTAs per SM the launch bounds promise (registers per thread <= 65536 / (256 MINB))
template <int NGC, int CW, bool XLO, bool BATCH, int MINB, bool EN = false>
__global__ void __launch_bounds__(kThreads, MINB) path_kernel(Args a) {
  constexpr int NG = CW * NGC;  // float4 granules per lane in warp-wide dots
  constexpr int CT = 32 * CW;   // chain threads (the first CW warps of CTA 0)
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ ChainSmem cs;
  __shared__ double dbuf[32];
  __shared__ int ibuf[32];
  __shared__ float fbuf[32];
  __shared__ int s_prob;

  // G CTAs cooperate on one problem: the whole grid, or a group of the batch
  const int G = BATCH ? a.gsize : (int)gridDim.x;
  const int cta = (int)blockIdx.x % G, grp = (int)blockIdx.x / G;
  char* wsb = a.ws + (BATCH ? (size_t)grp * a.cta_bytes : (size_t)0);
#define WS(T, name) reinterpret_cast<T*>(wsb + a.o_##name)
  Ctrl* ctl = WS(Ctrl, ctrl);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kThreads / 32;
  const int f0 = slice_begin(a, cta), f1 = slice_begin(a, cta + 1);
  // mask words of the slice: f0 is a multiple of 32 when the slice is not
  // empty; CTAs past the last feature (f0 == f1 == p) own no word
  const int wd0 = f0 >> 5, wd1 = f1 > f0 ? (f1 + 31) >> 5 : wd0;
  const int win_min = max(64, 4 * G * nwarps);  // smallest round window after a rollback
  ChainCtx cx{a.Xh,          a.Xl,           a.ldx,           a.ldw,          a.n,
                    a.ld4,         WS(int, A),     WS(int, chain),  WS(float4, ftab), WS(float2, bdf),
                    WS(float, nrmf), WS(ChainRec, recs), WS(float2, oldb), WS(float, snap), WS(float, msnap)};
  // dynamic shared memory of CTA 0: feature list of a round, then the column ring
  int* jl = reinterpret_cast<int*>(dsm);
  float4* ring = reinterpret_cast<float4*>(dsm + (((size_t)(a.s_cap + 1) * sizeof(int) + 127) & ~(size_t)127));
  unsigned* bc = &ctl->bar_count;
  unsigned* bg = &ctl->bar_gen;
  int* err = &ctl->err;
  const double u64 = 1.1102230246251565e-16;  // 2^-53
  const float bf = fp32_bound_factor<NG, XLO>();
  float bfc = bf;  // bound factor of the current check's c~
  float4 rh[NGC], rl[NGC];  // chain registers (CTA 0)
  long long tprof = clock64();
  // phase counters: thread 0 of CTA 0 (single path) or of every CTA (batched,
  // the counters of the problem it solved last)
  const bool prof_thread = cta == 0 && tid == 0;
#define PROF(k)                                   \
  do {                                            \
    if (prof_thread) {                            \
      const long long now_ = clock64();           \
      ctl->prof[k] += (unsigned long long)(now_ - tprof); \
      tprof = now_;                               \
    }                                             \
  } while (0)

#define GSYNC()                                            \
  do {                                                     \
    if (!grid_sync(bc, bg, err, (unsigned)G)) goto fail;   \
  } while (0)

  for (int it = 0;; ++it) {
    int b = 0;
    if (BATCH) {
      if (G == 1) {
        if (tid == 0) s_prob = atomicAdd(a.queue, 1);
        __syncthreads();
        b = s_prob;
        __syncthreads();
      } else {
        // CTA 0 of the group takes the problem and resets the fields the
        // set-up accumulates into; the group barrier publishes both
        if (cta == 0 && tid == 0) {
          ctl->err = 0;
          ctl->nonfinite = 0;
          ctl->m_bits = 0ull;
          ctl->mlo_bits = 0u;
          ctl->nzl = 0;
          ctl->prob = atomicAdd(a.queue, 1);
        }
        if (!grid_sync(bc, bg, err, (unsigned)G)) break;
        b = vload(ctl->prob);
      }
      if (b >= a.B) break;
      if (a.lockstep) {
        // this problem's own region carries its state from launch to launch
        wsb = a.ws + (size_t)b * a.cta_bytes;
        ctl = WS(Ctrl, ctrl);
        bc = &ctl->bar_count;
        bg = &ctl->bar_gen;
        err = &ctl->err;
        cx = ChainCtx{a.Xh,          a.Xl,           a.ldx,           a.ldw,            a.n,
                      a.ld4,         WS(int, A),     WS(int, chain),  WS(float4, ftab), WS(float2, bdf),
                      WS(float, nrmf), WS(ChainRec, recs), WS(float2, oldb), WS(float, snap), WS(float, msnap)};
        if (a.t0 == 0) {
          batch_setup<XLO>(a, ctl, wsb, b, dbuf, 0, a.p, true, true, true);
          if (tid == 0) ctl->failed = 0;
          __syncthreads();
        } else if (vload(ctl->failed) != 0) {
          continue;  // its records were stamped when it failed
        }
      } else if (G == 1) {
        batch_setup<XLO>(a, ctl, wsb, b, dbuf, 0, a.p, true, true, true);
      } else {
        // every CTA: the columns of its slice; CTA 0: y, rho and ||y||^2, then lambda_max
        batch_setup<XLO>(a, ctl, wsb, b, dbuf, f0, f1, false, cta == 0, false);
        if (!grid_sync(bc, bg, err, (unsigned)G)) goto fail;
        if (cta == 0) batch_setup<XLO>(a, ctl, wsb, b, dbuf, 0, 0, false, false, true);
        if (!grid_sync(bc, bg, err, (unsigned)G)) goto fail;
      }
      if (prof_thread && (!a.lockstep || a.t0 == 0)) {
        for (int k = 0; k < 8; ++k) ctl->prof[k] = 0ull;
        tprof = clock64();
      }
    } else if (it > 0) {
      break;
    }
    {
    const double* yv = BATCH ? WS(double, yb) : a.y;
    double* bout = a.beta_out + (size_t)b * a.T * a.p;
    uint32_t* mout = a.mask_out ? a.mask_out + (size_t)b * a.T * a.words : nullptr;
    lasso_path_stats* sout = a.stats + (size_t)b * a.T;
    const uint32_t rbits = BATCH ? chain_row_bits<NGC, CW>(a, b) : 0xffffffffu;
    if (vload(*err) != 0) goto fail;  // NaN/Inf input or lambda_max = 0

  const int t_begin = (BATCH && a.lockstep) ? a.t0 : 0, t_end = (BATCH && a.lockstep) ? a.t1 : a.T;
  for (int t = t_begin; t < t_end; ++t) {
    const double lam_path = __dmul_rn(vload(ctl->lambda_max), a.ratios[t]);
    // Elastic-Net (the paper's appendix): the Lasso with L1 weight a lambda on
    // the augmented design [X; sqrt(mu) I], [y; 0], mu = (1 - a) lambda.  The
    // augmented rows are never formed: the augmented residual's tail is
    // -sqrt(mu) beta, so x~_j^T rho~ = x_j^T rho - mu beta_j, ||x~_j||^2 =
    // ||x_j||^2 + mu, ||rho~||^2 = ||rho||^2 + mu ||beta||^2.  lam is the L1
    // weight everywhere below.
    const double lam = EN ? __dmul_rn(a.enet_alpha, lam_path) : lam_path;
    const double rdg = EN ? __dmul_rn(__dsub_rn(1.0, a.enet_alpha), lam_path) : 0.0;  // mu
    const float rdgf = __double2float_rn(rdg);
    // Elastic-Net: the extra FP32 forward error of a feature's ridge term when
    // c~ = fl(fl(x_j^T rho) - fl(mu beta_j)) (mu and beta_j's high part each
    // carry a relative 2^-24; the product and the difference are rounded once
    // each), cn being the adjusted c~; and the ridge term mu beta_j in FP64
    auto ridge_err = [&](int j, float cn) -> float {
      const float bh = ld_beta(cx, j).x;
      return bh != 0.f ? __fadd_ru(__fmul_ru(fabsf(__fmul_rn(rdgf, bh)), 4.8e-7f), __fmul_ru(fabsf(cn), 1.2e-7f))
                       : 0.f;
    };
    auto ridge_exact = [&](int j) -> double {
      const float2 b = ld_beta(cx, j);
      return __dmul_rn(rdg, __dadd_rn((double)b.x, (double)b.y));
    };
    // per-lambda table lambda / ||x_j||^2; full mask; optional restart
    for (int j = f0 + tid; j < f1; j += kThreads) {
      float4 tb = WS(float4, ftab)[j];
      if constexpr (EN) {
        // 1 / ||x~_j||^2 of the augmented column, for this lambda
        const double nr = __ldcg(WS(double, nrm) + j);
        const double den = __dadd_rn(__dmul_rn(nr, nr), rdg);
        const df2 iv = df_from_double(den > 0.0 ? __drcp_rn(den) : 0.0);
        tb.x = iv.h;
        tb.y = iv.l;
      }
      const df2 thr = df_from_double(__dmul_rn(lam, __dadd_rn((double)tb.x, (double)tb.y)));
      tb.z = thr.h;
      tb.w = thr.l;
      WS(float4, ftab)[j] = tb;
      if (t > 0 && !a.warm_start) WS(float2, bdf)[j] = WS(float2, b0df)[j];
    }
    for (int w = wd0 + tid; w < wd1; w += kThreads) {
      const int lo = w * 32, hi = min(a.p, lo + 32);
      WS(uint32_t, mask)[w] = (hi - lo == 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
    }
    if (cta == 0 && t > 0 && !a.warm_start)
      for (int i = tid; i < a.ldw; i += kThreads) {
        WS(float, rho_h)[i] = __ldcg(WS(float, rho0_h) + i);
        WS(float, rho_l)[i] = __ldcg(WS(float, rho0_l) + i);
      }
    long long epochs = 0, checks = 0, xcols = 0;
    int scope_n = a.p;  // X^T rho scope of the next check
    GSYNC();

    for (;;) {
      // ======================= CHECK =======================
      PROF(7);
      // (C1) ||rho||^2, y^T rho (every CTA), c~ for the slice, sum |beta| of the slice
      double rr = 0.0, yr = 0.0;
      for (int i = tid; i < a.n; i += kThreads) {
        const double r = __dadd_rn((double)__ldcg(WS(float, rho_h) + i), (double)__ldcg(WS(float, rho_l) + i));
        rr = __fma_rn(r, r, rr);
        yr = __fma_rn(yv[i], r, yr);
      }
      rr = block_sum_d(rr, dbuf);
      yr = block_sum_d(yr, dbuf);
      const float rnormf = __fmul_ru(__fsqrt_ru(__double2float_ru(rr)), 1.0001f);
      {
        float4 r4[NG];
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const int g = lane + 32 * k;
          r4[k] = (g < a.ld4) ? ldcg4(WS(float, rho_h), g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float mlo = 0.f;
        // the first check of a lambda of a lockstep batch takes c~ from the
        // batched tensor-core product, with its own error factor
        const bool from_gemm = BATCH && a.cfirst != nullptr && checks == 0;
        bfc = from_gemm ? a.cfactor : bf;
        for (int j = f0 + warp; j < f1; j += nwarps) {
          const bool in = a.xtr_scope == 0 || ((__ldcg(WS(uint32_t, mask) + (j >> 5)) >> (j & 31)) & 1u);
          float c = 0.f;
          if (in) {
            c = from_gemm ? __ldcg(a.cfirst + (size_t)j + (size_t)b * a.ldc)
                          : warp_dot_f32<NG>(a.Xh + (long long)j * a.ldx, r4, a.ld4, a.n);
            float E = __fmul_ru(__fmul_ru(bfc, __ldcg(WS(float, nrmf) + j)), rnormf) + 1e-37f;
            if constexpr (EN) {
              const float bh = ld_beta(cx, j).x;
              if (bh != 0.f) c = __fsub_rn(c, __fmul_rn(rdgf, bh));  // x~_j^T rho~
              E = __fadd_ru(E, ridge_err(j, c));
            }
            mlo = fmaxf(mlo, __fsub_rd(fabsf(c), E));
          }
          if (lane == 0) WS(float, ctil)[j] = c;
        }
        if (lane == 0) atomicMax(&ctl->mlo_bits, __float_as_uint(fmaxf(mlo, 0.f)));
        double l1p = 0.0, l2p = 0.0;
        for (int j = f0 + tid; j < f1; j += kThreads) {
          const float2 b = ld_beta(cx, j);
          const double bv = __dadd_rn((double)b.x, (double)b.y);
          l1p = __dadd_rn(l1p, fabs(bv));
          if constexpr (EN) l2p = __fma_rn(bv, bv, l2p);
        }
        l1p = block_sum_d(l1p, dbuf);
        if (tid == 0) WS(double, part_l1)[cta] = l1p;
        if constexpr (EN) {
          l2p = block_sum_d(l2p, dbuf);
          if (tid == 0) WS(double, part_l2)[cta] = l2p;
        }
      }
      GSYNC();
      // (C2) exact refinement of the candidates for the maximum
      {
        const float mlo = __uint_as_float(vload(ctl->mlo_bits));
        for (int j = f0 + warp; j < f1; j += nwarps) {
          const bool in = a.xtr_scope == 0 || ((__ldcg(WS(uint32_t, mask) + (j >> 5)) >> (j & 31)) & 1u);
          if (!in) continue;
          const float c = __ldcg(WS(float, ctil) + j);
          const float nf = __ldcg(WS(float, nrmf) + j);
          float E = __fmul_ru(__fmul_ru(bfc, nf), rnormf) + 1e-37f;
          if constexpr (EN) E = __fadd_ru(E, ridge_err(j, c));
          if (__fadd_ru(fabsf(c), E) >= mlo) {
            const df2 ce = warp_dot_exact<NG, XLO>(cx, j, WS(float, rho_h), WS(float, rho_l), __fmul_ru(nf, rnormf));
            double cv = df_to_double(ce);
            if constexpr (EN) cv = __dsub_rn(cv, ridge_exact(j));
            cv = fabs(cv);
            if (lane == 0) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(cv));
          }
        }
      }
      GSYNC();
      // (C3) objectives, gap, radius (identical in every CTA); sphere test on the slice
      double l1 = 0.0;
      for (int c = tid; c < G; c += kThreads) l1 = __dadd_rn(l1, __ldcg(WS(double, part_l1) + c));
      l1 = block_sum_d(l1, dbuf);
      double l2 = 0.0;
      if constexpr (EN) {
        // ||rho~||^2 = ||rho||^2 + mu ||beta||^2
        for (int c = tid; c < G; c += kThreads) l2 = __dadd_rn(l2, __ldcg(WS(double, part_l2) + c));
        l2 = block_sum_d(l2, dbuf);
        rr = __dadd_rn(rr, __dmul_rn(rdg, l2));
      }
      const double m = __longlong_as_double((long long)vload(ctl->m_bits));
      double alpha;
      if (a.dual_point == 0) {
        alpha = __drcp_rn(lam > m ? lam : m);
      } else if (rr == 0.0) {
        alpha = 0.0;
      } else {
        double al = __ddiv_rn(yr, __dmul_rn(lam, rr));
        if (m > 0.0) {
          const double lim = __drcp_rn(m);
          if (al < -lim) al = -lim;
          if (al > lim) al = lim;
        }
        alpha = al;
      }
      double d2 = 0.0;
      for (int i = tid; i < a.n; i += kThreads) {
        const double r = __dadd_rn((double)__ldcg(WS(float, rho_h) + i), (double)__ldcg(WS(float, rho_l) + i));
        const double dd = __dsub_rn(__dmul_rn(lam, __dmul_rn(alpha, r)), yv[i]);
        d2 = __fma_rn(dd, dd, d2);
      }
      d2 = block_sum_d(d2, dbuf);
      if constexpr (EN) {
        // the augmented rows: (lambda alpha (-sqrt(mu) beta_j))^2
        const double la = __dmul_rn(lam, alpha);
        d2 = __dadd_rn(d2, __dmul_rn(__dmul_rn(la, la), __dmul_rn(rdg, l2)));
      }
      const double yy = vload(ctl->yy);
      const double P = __dadd_rn(__dmul_rn(0.5, rr), __dmul_rn(lam, l1));
      const double D = __dsub_rn(__dmul_rn(0.5, yy), __dmul_rn(0.5, d2));
      const double Gap = __dsub_rn(P, D);
      const double tau = 2.0 * (double)(a.n + a.p + (EN ? a.p : 0) + 8) * u64 * (rr + lam * l1 + yy + d2);
      const double Gs = (Gap > 0.0 ? Gap : 0.0) + tau;
      double rad = __ddiv_rn(__dsqrt_rn(__dmul_rn(2.0, Gs)), lam);
      if (a.refined_radius == 1) {
        // Thm. 2's radius (R^2 - r(beta)^2)^(1/2): sqrt(2 G)/lambda, or R =
        // ||theta - y/lambda|| when the clipped r(beta) is 0 (P > ||y||^2/2)
        const double Rt = __ddiv_rn(__dsqrt_rn(__dadd_rn(d2, tau)), lam);
        if (Rt < rad) rad = Rt;
      }
      const double aa = fabs(alpha);
      // GAP SAFE dome (Eq. (11), parameters of the appendix): center
      // (y/lambda + theta)/2, radius R/2 with R = ||y/lambda - theta||, unit
      // normal (y/lambda - theta)/R, ratio 2 r^2/R^2 - 1 with r the radius of
      // Thm. 2 from the primal point; lambda^2 R^2 is enlarged and lambda^2 r^2
      // reduced by the rounding bound tau, as the sphere's gap is.  When
      // theta = y/lambda the dome is a point and only the sphere runs.
      const bool dome = a.screen_rule == 1 && d2 > 0.0;
      double drad = 0.0, dal = 0.0, dR = 1.0;
      if (dome) {
        const double big = __dadd_rn(d2, tau);
        double small = __dsub_rn(__dsub_rn(yy, __dmul_rn(2.0, P)), tau);
        if (small < 0.0) small = 0.0;
        double q = __ddiv_rn(small, big);
        if (q > 1.0) q = 1.0;
        dal = __dsub_rn(__dmul_rn(2.0, q), 1.0);
        drad = __ddiv_rn(__dmul_rn(0.5, __dsqrt_rn(big)), lam);
        dR = __ddiv_rn(__dsqrt_rn(d2), lam);
      }
      ++checks;
      xcols += scope_n;
      const bool stop = Gap <= vload(ctl->eps);
      const bool cap = epochs >= a.max_epochs;
      {
        const float aaf_lo = __double2float_rd(aa), aaf_hi = __double2float_ru(aa);
        const float radf_lo = __double2float_rd(rad), radf_hi = __double2float_ru(rad);
        int kept = 0, sup = 0, nnz = 0, zero = 0;
        // each warp handles 32 consecutive features = one mask word
        for (int w0 = f0 + 32 * warp; w0 < f1; w0 += 32 * nwarps) {
          const int j = w0 + lane;
          const bool valid = j < f1;
          const uint32_t word = __ldcg(WS(uint32_t, mask) + (w0 >> 5));
          const bool was = valid && ((word >> lane) & 1u);
          bool keep = was, amb = false;
          if (was) {
            const float c = __ldcg(WS(float, ctil) + j);
            const float nf = __ldcg(WS(float, nrmf) + j);
            float E = __fmul_ru(__fmul_ru(bfc, nf), rnormf) + 1e-37f;
            float nfl = __double2float_rd(__ldcg(WS(double, nrm) + j));
            float nfr = nf;  // ||x~_j|| rounded up: the radius term's norm
            if constexpr (EN) {
              E = __fadd_ru(E, ridge_err(j, c));
              nfr = __fsqrt_ru(__fadd_ru(__fmul_ru(nf, nf), __double2float_ru(rdg)));
              nfl = __fsqrt_rd(__fadd_rd(__fmul_rd(nfl, nfl), __double2float_rd(rdg)));
            }
            // rigorous FP32 brackets of mu_j = |c_j| |alpha| + r ||x_j||
            const float mu_hi = __fadd_ru(__fmul_ru(__fadd_ru(fabsf(c), E), aaf_hi), __fmul_ru(radf_hi, nfr));
            const float clo = fmaxf(__fsub_rd(fabsf(c), E), 0.f);
            const float mu_lo = __fadd_rd(__fmul_rd(clo, aaf_lo), __fmul_rd(radf_lo, nfl));
            // a feature the sphere screens for certain is screened by the
            // dome too (the dome lies inside the sphere); any other one gets
            // the exact evaluation when the dome runs
            if (mu_hi < 0.999999f) keep = false;
            else if (mu_lo >= 1.000001f && !dome) keep = true;
            else amb = true;
          }
          // exact decision for the undecided ones, as the FP64 tests of
          // Eq. (7) (sphere) and Eq. (11) (dome)
          unsigned ambm = __ballot_sync(0xffffffffu, amb);
          while (ambm) {
            const int l = __ffs(ambm) - 1;
            ambm &= ambm - 1;
            const int jj = w0 + l;
            const df2 ce = warp_dot_exact<NG, XLO>(cx, jj, WS(float, rho_h), WS(float, rho_l), __fmul_ru(__ldcg(WS(float, nrmf) + jj), rnormf));
            double cj = df_to_double(ce), xn = __ldcg(WS(double, nrm) + jj);
            if constexpr (EN) {
              cj = __dsub_rn(cj, ridge_exact(jj));
              xn = __dsqrt_rn(__dadd_rn(__dmul_rn(xn, xn), rdg));
            }
            const double mu = __dadd_rn(__dmul_rn(fabs(cj), aa), __dmul_rn(rad, xn));
            bool kp = !(mu < 1.0);
            if (dome) {
              const double xt = __dmul_rn(alpha, cj);                       // x_j^T theta
              const double xy = __ddiv_rn(__ldcg(WS(double, cy) + jj), lam);  // x_j^T y / lambda
              const double xc = __dmul_rn(0.5, __dadd_rn(xy, xt));          // x_j^T center
              const double xnr = __ddiv_rn(__dsub_rn(xy, xt), dR);          // x_j^T normal
              const double md = fmax(dome_support(xc, drad, dal, xnr, xn), dome_support(-xc, drad, dal, -xnr, xn));
              if (md < 1.0) kp = false;
            }
            if (lane == l) keep = kp;
          }
          const float2 bj = valid ? ld_beta(cx, j) : make_float2(0.f, 0.f);
          bool nz = nonzero2(bj);
          // a newly screened nonzero coefficient is set to zero when the
          // solver goes on (Remark 3); its residual share is added back by CTA 0
          const bool zeroed = was && !keep && nz && !stop && !cap;
          if (zeroed) {
            WS(double, zl_b)[j] = __dadd_rn((double)bj.x, (double)bj.y);
            WS(float2, bdf)[j] = make_float2(0.f, 0.f);
            nz = false;
          }
          const uint32_t zw = __ballot_sync(0xffffffffu, zeroed);
          zero += __popc(zw);
          const uint32_t nwd = __ballot_sync(0xffffffffu, keep);
          if (lane == 0) {
            WS(uint32_t, mask)[w0 >> 5] = nwd;
            WS(uint32_t, zbits)[w0 >> 5] = zw;
          }
          kept += __popc(nwd);
          sup += __popc(__ballot_sync(0xffffffffu, keep && nz));
          nnz += __popc(__ballot_sync(0xffffffffu, valid && nz));
        }
        if (lane != 0) kept = sup = nnz = zero = 0;
        kept = block_sum_i(kept, ibuf);
        sup = block_sum_i(sup, ibuf);
        nnz = block_sum_i(nnz, ibuf);
        zero = block_sum_i(zero, ibuf);
        if (tid == 0) {
          WS(int, cnt_kept)[cta] = kept;
          WS(int, cnt_sup)[cta] = sup;
          WS(int, cnt_nnz)[cta] = nnz;
          WS(int, cnt_zero)[cta] = zero;
        }
      }
      GSYNC();
      // (C4) totals and this CTA's offsets; the maxima are reset for the next check
      int totk = 0, tots = 0, totn = 0, totz = 0, pk = 0, ps = 0, pz = 0;
      for (int c = tid; c < G; c += kThreads) {
        const int k = __ldcg(WS(int, cnt_kept) + c), s = __ldcg(WS(int, cnt_sup) + c), z = __ldcg(WS(int, cnt_zero) + c);
        totk += k;
        tots += s;
        totz += z;
        totn += __ldcg(WS(int, cnt_nnz) + c);
        if (c < cta) {
          pk += k;
          ps += s;
          pz += z;
        }
      }
      totk = block_sum_i(totk, ibuf);
      tots = block_sum_i(tots, ibuf);
      totn = block_sum_i(totn, ibuf);
      totz = block_sum_i(totz, ibuf);
      pk = block_sum_i(pk, ibuf);
      ps = block_sum_i(ps, ibuf);
      pz = block_sum_i(pz, ibuf);
      if (cta == 0 && tid == 0) {
        ctl->m_bits = 0ull;
        ctl->mlo_bits = 0u;
      }
      if (stop || cap) {
        // outputs of this lambda
        for (int j = f0 + tid; j < f1; j += kThreads) {
          const float2 b = ld_beta(cx, j);
          bout[(long long)t * a.p + j] = __dadd_rn((double)b.x, (double)b.y);
        }
        if (mout)
          for (int w = wd0 + tid; w < wd1; w += kThreads)
            mout[(long long)t * a.words + w] = __ldcg(WS(uint32_t, mask) + w);
        if (cta == 0 && tid == 0) {
          lasso_path_stats st;
          st.lambda = lam_path;
          st.primal = P;
          st.dual = D;
          st.gap = Gap;
          st.radius = rad;
          st.alpha = alpha;
          st.epochs = epochs;
          st.checks = checks;
          st.n_active = totk;
          st.n_nonzero = totn;
          st.x_columns = xcols;
          st.converged = stop ? 1 : 0;
          st.status = stop ? kStatusOK : kStatusNotConverged;
          sout[t] = st;
        }
        GSYNC();
        break;
      }
      // compaction: ascending safe-active list A, support positions sup0 and
      // the ascending list of coefficients the check set to zero.  Each warp
      // takes a contiguous run of the slice's mask words: count, prefix over
      // the warps, write.
      {
        const int w_first = wd0, w_last = wd1;
        const int nwd = w_last - w_first, per = (nwd + nwarps - 1) / nwarps;
        const int wb = w_first + warp * per, we = min(w_last, wb + per);
        int ck = 0, cs_ = 0, cz = 0;
        for (int w = wb; w < we; ++w) {
          const uint32_t word = __ldcg(WS(uint32_t, mask) + w);
          const int j = w * 32 + lane;
          const bool keep = (word >> lane) & 1u;
          const bool nz = keep && nonzero2(ld_beta(cx, j));
          ck += __popc(word);
          cs_ += __popc(__ballot_sync(0xffffffffu, nz));
          cz += __popc(__ldcg(WS(uint32_t, zbits) + w));
        }
        __syncthreads();
        if (lane == 0) {
          ibuf[warp] = ck;
          ibuf[8 + warp] = cs_;
          ibuf[16 + warp] = cz;
        }
        __syncthreads();
        int runk = pk, runs = ps, runz = pz;
        for (int w = 0; w < warp; ++w) {
          runk += ibuf[w];
          runs += ibuf[8 + w];
          runz += ibuf[16 + w];
        }
        __syncthreads();
        const float lam_lo = __fmul_rd(__double2float_rd(lam), 1.0f - 1e-6f);
        for (int w = wb; w < we; ++w) {
          const int j = w * 32 + lane;
          const uint32_t word = __ldcg(WS(uint32_t, mask) + w);
          const uint32_t zw = __ldcg(WS(uint32_t, zbits) + w);
          const bool keep = (word >> lane) & 1u;
          const bool nz = keep && nonzero2(ld_beta(cx, j));
          const unsigned lower = (1u << lane) - 1u;
          const int kpos = runk + __popc(word & lower);
          const unsigned smk = __ballot_sync(0xffffffffu, nz);
          if (keep) {
            // certificate of a zero coefficient: slack / ||x_j|| with
            // slack <= lambda - |x_j^T rho| (the check's c~ and its bound);
            // nonzero coefficients are chain entries (never verified)
            float sk = kSkChain;
            if (!nz) {
              const float nf = __ldcg(WS(float, nrmf) + j);
              const float E = __fmul_ru(__fmul_ru(bfc, nf), rnormf) + 1e-37f;
              const float slack = __fsub_rd(lam_lo, __fadd_ru(fabsf(__ldcg(WS(float, ctil) + j)), E));
              sk = (slack > 0.f && nf > 0.f) ? __fdiv_rd(slack, nf) : kSkNone;
            }
            WS(float, sk)[kpos] = sk;
            WS(float, mref)[kpos] = 0.f;
            WS(int, A)[kpos] = j;
          }
          if (nz) WS(int, sup0)[runs + __popc(smk & lower)] = kpos;
          if ((zw >> lane) & 1u) WS(int, zl_j)[runz + __popc(zw & lower)] = j;
          runk += __popc(word);
          runs += __popc(smk);
          runz += __popc(zw);
        }
      }
      if (cta == 0 && tid == 0) {
        ctl->q = totk;
        ctl->s = tots;
        ctl->nzl = totz;
        ctl->mcur = 0.f;
        ctl->win = totk;
      }
      scope_n = a.xtr_scope == 0 ? a.p : totk;
      GSYNC();
      PROF(0);
      // ======================= PASSES =======================
      {
        const int q = vload(ctl->q);
        int s = vload(ctl->s);
        int* sup = WS(int, sup0);
        int* sup_next = WS(int, sup1);
        if (cta == 0) {
          // residual shares of the coefficients removed by the check, ascending j
          const int nz = vload(ctl->nzl);
          if (nz > 0) {
            load_rho_regs<NGC, CW>(cx, WS(float, rho_h), WS(float, rho_l), rh, rl);
            for (int i = 0; i < nz; ++i) {
              const int jj = __ldcg(WS(int, zl_j) + i);
              const df2 d = df_from_double(-__ldcg(WS(double, zl_b) + jj));  // rho -= (0 - b) x_j
              const float* col = a.Xh + (long long)jj * a.ldx;
              const float* coll = XLO ? a.Xl + (long long)jj * a.ldx : nullptr;
#pragma unroll
              for (int k = 0; k < NGC; ++k) {
                const int g = tid + CT * k;
                if (tid < CT && g < a.ld4) {
                  const float4 x = mask_bits(ld_x4(col, g, a.n), rbits >> (4 * k));
                  if (XLO) {
                    const float4 xl = mask_bits(ld_x4(coll, g, a.n), rbits >> (4 * k));
                    axpy_df2(x.x, xl.x, d.h, d.l, rh[k].x, rl[k].x);
                    axpy_df2(x.y, xl.y, d.h, d.l, rh[k].y, rl[k].y);
                    axpy_df2(x.z, xl.z, d.h, d.l, rh[k].z, rl[k].z);
                    axpy_df2(x.w, xl.w, d.h, d.l, rh[k].w, rl[k].w);
                  } else {
                    axpy_df(x.x, d.h, d.l, rh[k].x, rl[k].x);
                    axpy_df(x.y, d.h, d.l, rh[k].y, rl[k].y);
                    axpy_df(x.z, d.h, d.l, rh[k].z, rl[k].z);
                    axpy_df(x.w, d.h, d.l, rh[k].w, rl[k].w);
                  }
                }
              }
            }
            store_rho_regs<NGC, CW>(cx, WS(float, rho_h), WS(float, rho_l), rh, rl);
            __syncthreads();
            if (tid == 0) {
              float mv = ctl->mcur;
              for (int i = 0; i < nz; ++i) {
                const int jj = __ldcg(WS(int, zl_j) + i);
                mv = __fadd_ru(mv, __fmul_ru(__double2float_ru(fabs(__ldcg(WS(double, zl_b) + jj))),
                                             __ldcg(WS(float, nrmf) + jj)));
              }
              ctl->mcur = mv;
              ctl->nzl = 0;
            }
          }
        }
        for (int e = 0; e < a.f && epochs < a.max_epochs; ++e) {
          // ---- one pass over the safe-active list, in rounds
          if (cta == 0) {
            load_rho_regs<NGC, CW>(cx, WS(float, rho_h), WS(float, rho_l), rh, rl);
            if (tid == 0) {
              ctl->pos = 0;
              ctl->sup_idx = 0;
              ctl->forced = -1;
              ctl->n_entered = 0;
            }
            __syncthreads();
          }
          for (;;) {
            PROF(7);
            // R1 (CTA 0): chain = [forced entry] + the support positions of the
            // round's window [pos, pos + win) (at most s_cap of them).  The round
            // ends at the window's end, or at the first support position left out.
            if (cta == 0) {
              const int si = vload(ctl->sup_idx), forced = vload(ctl->forced);
              const int pos0 = vload(ctl->pos);
              const int plim = (int)min((long long)q, (long long)pos0 + vload(ctl->win));
              const int in_win = lower_bound_i(sup + si, s - si, plim);
              const int take = min(in_win, a.s_cap - (forced >= 0 ? 1 : 0));
              const int nc = take + (forced >= 0 ? 1 : 0);
              const int next = (si + take < s) ? __ldcg(sup + si + take) : q;
              const int rend = take < in_win ? next : min(plim, next);
              for (int c = tid; c < nc; c += kThreads)
                WS(int, chain)[c] = (forced >= 0) ? (c == 0 ? forced : __ldcg(sup + si + c - 1)) : __ldcg(sup + si + c);
              __syncthreads();
              const float rb = rho_bound_from_regs<NGC, EN>(cx, rh, lam, nc, fbuf, rdg);
              if (tid == 0) {
                ctl->rho_bound = rb;
                ctl->nc = nc;
                ctl->round_end = rend;
                ctl->fstar = kNoPos;
                WS(float, msnap)[0] = ctl->mcur;
              }
              store_rho_regs<NGC, CW>(cx, WS(float, snap), WS(float, snap) + a.ldw, rh, rl);  // snapshot 0
              __syncthreads();
              run_chain<NGC, CW, XLO, EN>(cx, cs, ring, jl, nc, rb, rh, rl, rbits, df_from_double(rdg));
              __threadfence();
              if (prof_thread) ctl->prof[5] += (unsigned long long)nc;
            }
            PROF(1);
            GSYNC();
            // R2 (all CTAs): the zero coefficients of [pos, round_end) must stay zero
            {
              const int pos = vload(ctl->pos), rend = vload(ctl->round_end), nc = vload(ctl->nc);
              const float rb = vload(ctl->rho_bound);
              const int span = rend - pos;
              const int gw = cta * nwarps + warp, nwg = G * nwarps;
              const int chunk = (span + nwg - 1) / nwg;
              const int i0 = pos + gw * chunk, i1 = min(rend, i0 + chunk);
              if (span > 0 && i0 < i1) {
                // a zero coefficient whose certificate survives the movement of
                // the residual since it was issued stays zero without a read:
                // |x_j^T rho| <= lambda - slack + ||x_j|| (M_now - M_ref) < lambda
                const float mend = __ldcg(WS(float, msnap) + nc);
                const float* skp = WS(float, sk);
                float* mrp = WS(float, mref);
                int seg = lower_bound_i(WS(int, chain), nc, i0);
                float4 r4[NG];
                int loaded = -1;
                const float lamf = __double2float_rn(lam);
                const float lam_lo = __fmul_rd(__double2float_rd(lam), 1.0f - 1e-6f);
                bool stop_warp = false;
                for (int base = i0; base < i1 && !stop_warp; base += 32) {
                  const int il = base + lane;
                  bool need = false;
                  if (il < i1) {
                    const float sk = __ldcg(skp + il);
                    need = !(__fsub_ru(mend, __ldcg(mrp + il)) < sk);
                  }
                  unsigned needm = __ballot_sync(0xffffffffu, need);
                  // the verdict for position i from its FP32 correlation c with the
                  // snapshot sh: stays zero (certificate renewed) or enters
                  auto decide = [&](int i, int j, float c, const float* sh) -> bool {
                    const float nf = __ldcg(WS(float, nrmf) + j);
                    const float E = __fmul_ru(__fmul_ru(bf, nf), rb) + 1e-37f;
                    bool enters;
                    if (__fadd_ru(fabsf(c), E) < lamf * (1.0f - 1e-6f)) enters = false;
                    else if (__fsub_rd(fabsf(c), E) > lamf * (1.0f + 1e-6f)) enters = true;
                    else {
                      const df2 g = warp_dot_exact<NG, XLO>(cx, j, sh, sh + a.ldw, __fmul_ru(nf, rb));
                      df2 nb, d;
                      cd_update(g, df2{0.f, 0.f}, __ldcg(WS(float4, ftab) + j), nb, d);
                      enters = !df_is_zero(d);
                    }
                    if (enters) {
                      if (lane == 0) atomicMin(&ctl->fstar, i);
                    } else if (lane == 0) {
                      const float slack = __fsub_rd(lam_lo, __fadd_ru(fabsf(c), E));
                      WS(float, sk)[i] = (slack > 0.f && nf > 0.f) ? __fdiv_rd(slack, nf) : kSkNone;
                      mrp[i] = __ldcg(WS(float, msnap) + seg);
                    }
                    return enters;
                  };
                  while (needm) {
                    const int i = base + __ffs(needm) - 1;
                    needm &= needm - 1;
                    // fstar moves under other warps' atomicMin: one lane reads it
                    // so that the whole warp takes the same branch before the
                    // full-mask dot products below
                    if (i > __shfl_sync(0xffffffffu, vload(ctl->fstar), 0)) {
                      stop_warp = true;
                      break;
                    }
                    while (seg < nc && __ldcg(WS(int, chain) + seg) < i) ++seg;
                    const float* sh = WS(float, snap) + (size_t)seg * 2 * a.ldw;
                    if (loaded != seg) {
#pragma unroll
                      for (int k = 0; k < NG; ++k) {
                        const int g = lane + 32 * k;
                        r4[k] = (g < a.ld4) ? ldcg4(sh, g) : make_float4(0.f, 0.f, 0.f, 0.f);
                      }
                      loaded = seg;
                    }
                    const int j = __ldcg(WS(int, A) + i);
                    // the next needed position shares the snapshot when no chain
                    // entry lies between them: verify both with one pass of loads
                    // (up to 8 granules per lane; longer columns keep one)
                    constexpr bool kPair = NG <= 8;
                    const int seg_end = seg < nc ? __ldcg(WS(int, chain) + seg) : 0x7fffffff;
                    const int i2 = needm ? base + __ffs(needm) - 1 : 0x7fffffff;
                    if (kPair && i2 < seg_end) {
                      const int j2 = __ldcg(WS(int, A) + i2);
                      float c, c2;
                      warp_dot_f32_2<NG>(a.Xh + (long long)j * a.ldx, a.Xh + (long long)j2 * a.ldx, r4, a.ld4, a.n,
                                         c, c2);
                      if (decide(i, j, c, sh)) {
                        stop_warp = true;
                        break;
                      }
                      needm &= needm - 1;
                      if (decide(i2, j2, c2, sh)) {
                        stop_warp = true;
                        break;
                      }
                    } else {
                      const float c = warp_dot_f32<NG>(a.Xh + (long long)j * a.ldx, r4, a.ld4, a.n);
                      if (decide(i, j, c, sh)) {
                        stop_warp = true;
                        break;
                      }
                    }
                  }
                }
              }
            }
            GSYNC();
            PROF(2);
            // R3 (CTA 0): accept the round, or roll back to the first entering position
            if (cta == 0) {
              const int fst = vload(ctl->fstar), nc = vload(ctl->nc), rend = vload(ctl->round_end);
              const int forced = vload(ctl->forced), si = vload(ctl->sup_idx);
              if (fst == kNoPos) {
                if (tid == 0) {
                  if (forced >= 0) {
                    if (nonzero2(ld_beta(cx, __ldcg(WS(int, A) + forced)))) WS(int, entered)[ctl->n_entered++] = forced;
                    else WS(float, sk)[forced] = kSkNone;  // stayed zero: verify it next pass
                  }
                  ctl->mcur = __ldcg(WS(float, msnap) + nc);
                  ctl->sup_idx = si + nc - (forced >= 0 ? 1 : 0);
                  ctl->pos = rend;
                  ctl->forced = -1;
                  ctl->done = rend >= q ? 1 : 0;
                  ctl->win = (int)min((long long)q, 2ll * vload(ctl->win));
                }
              } else {
                // chain entries before the entering position stand; later ones are undone
                if (prof_thread) ctl->prof[6] += 1ull;
                const int seg = lower_bound_i(WS(int, chain), nc, fst);
                for (int c = seg + tid; c < nc; c += kThreads) WS(float2, bdf)[__ldcg(WS(int, A) + __ldcg(WS(int, chain) + c))] = WS(float2, oldb)[c];
                const float* sh = WS(float, snap) + (size_t)seg * 2 * a.ldw;
                load_rho_regs<NGC, CW>(cx, sh, sh + a.ldw, rh, rl);
                __syncthreads();
                if (tid == 0) {
                  if (forced >= 0) {
                    if (nonzero2(ld_beta(cx, __ldcg(WS(int, A) + forced)))) WS(int, entered)[ctl->n_entered++] = forced;
                    else WS(float, sk)[forced] = kSkNone;
                  }
                  WS(float, sk)[fst] = kSkChain;  // the next round's forced chain entry
                  // certificates issued on the undone branch stay valid if the
                  // counter also pays for the way back: from any point e of
                  // that branch, ||rho_t - rho_e|| <= (M_e - M_seg) + (new
                  // movement) <= (2 M_end - M_seg - M_e) + (new movement)
                  const float m_end = __ldcg(WS(float, msnap) + nc), m_seg = __ldcg(WS(float, msnap) + seg);
                  ctl->mcur = __fsub_ru(__fmul_ru(2.0f, m_end), m_seg);
                  // the verification beyond fst was spent on an undone branch: the
                  // next window is twice the span this round kept, and at least
                  // four positions per warp of the grid
                  const int pos_r = vload(ctl->pos);
                  ctl->win = max(win_min, 2 * (fst - pos_r));
                  ctl->sup_idx = si + seg - (forced >= 0 ? 1 : 0);
                  ctl->forced = fst;
                  ctl->pos = fst;
                  ctl->done = 0;
                }
              }
              __threadfence();
              __syncthreads();
            }
            GSYNC();
            PROF(3);
            if (vload(ctl->done)) break;
          }
          // end of pass (CTA 0): write rho; next support list = survivors of the
          // old list merged with the entered positions (both ascending)
          if (cta == 0) {
            store_rho_regs<NGC, CW>(cx, WS(float, rho_h), WS(float, rho_l), rh, rl);
            const int ne = vload(ctl->n_entered);
            __syncthreads();
            int nsurv = 0;
            for (int base = 0; base < s; base += kThreads) {
              const int i = base + tid;
              int posv = 0;
              bool keep = false;
              if (i < s) {
                posv = __ldcg(sup + i);
                keep = nonzero2(ld_beta(cx, __ldcg(WS(int, A) + posv)));
                if (!keep) WS(float, sk)[posv] = kSkNone;  // left the support: a zero coefficient now
              }
              int tot;
              const int r = block_rank(keep, ibuf, &tot);
              if (keep) WS(int, zl_j)[nsurv + r] = posv;
              nsurv += tot;
            }
            __syncthreads();
            for (int k = tid; k < nsurv; k += kThreads) {
              const int v = __ldcg(WS(int, zl_j) + k);
              sup_next[k + lower_bound_i(WS(int, entered), ne, v)] = v;
            }
            for (int k = tid; k < ne; k += kThreads) {
              const int v = __ldcg(WS(int, entered) + k);
              sup_next[k + lower_bound_i(WS(int, zl_j), nsurv, v)] = v;
            }
            if (tid == 0) ctl->s = nsurv + ne;
            __threadfence();
            __syncthreads();
          }
          ++epochs;
          xcols += q;
          GSYNC();
          PROF(4);
          s = vload(ctl->s);
          int* tmp = sup;
          sup = sup_next;
          sup_next = tmp;
        }
      }
      GSYNC();
    }
  }  // lambda loop
    }
    continue;
  fail:
    // a device error on this problem (NaN/Inf input, lambda_max = 0, a wait
    // that timed out): the single-path launch stops here (the records are
    // stamped by stats_error_kernel); a batched CTA stamps this problem's
    // records and moves on to the next problem
    if (!BATCH) break;
    {
      const int e = vload(*err);
      // a group: every CTA has read the code before CTA 0 clears it (this
      // barrier completes although it reports the pending error)
      if (G > 1) grid_sync(bc, bg, err, (unsigned)G);
      if (cta == 0) {
        lasso_path_stats* so = a.stats + (size_t)b * a.T;
        const int tf0 = a.lockstep ? a.t0 : 0;
        for (int t = tf0 + tid; t < a.T; t += kThreads) {
          lasso_path_stats st{};
          st.lambda = vload(ctl->lambda_max) * a.ratios[t];
          st.status = e;
          so[t] = st;
        }
        for (size_t k = (size_t)tf0 * a.p + tid; k < (size_t)a.T * a.p; k += kThreads)
          a.beta_out[(size_t)b * a.T * a.p + k] = 0.0;
        __syncthreads();
        if (tid == 0) {
          ctl->err = 0;
          ctl->failed = e;
        }
        __syncthreads();
      }
      // after a timed-out wait the group's barrier may be out of step: the
      // group stops, and the other groups take the remaining problems
      if (G > 1 && e == kErrTimeout) break;
    }
  }
#undef GSYNC
#undef PROF
#undef WS
}

// ---------------------------------------------------------------- setup kernels
// ||x_j||, 1/||x_j||^2, c0_j = x_j^T y -> lambda_max = ||X^T y||_inf (Sec. 1.2),
// finiteness of X, split planes of an FP64 X, beta0 in double-float.  c0 is
// kept for the dome test.
template <typename XT>
__global__ void precompute_kernel(const XT* X, long long ldx, int n, int p, const double* y, const double* beta0,
                                  float* Xh, float* Xl, long long ldh, double* nrm, float* nrmf, float4* ftab,
                                  float2* bdf, float2* b0df, double* cy, Ctrl* ctl) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < p; j += nwarps) {
    const XT* col = X + (long long)j * ldx;
    double s2 = 0.0, sy = 0.0;
    bool finite = true;
    for (int i = lane; i < n; i += 32) {
      const double x = (double)col[i];
      finite = finite && isfinite(x);
      s2 = __fma_rn(x, x, s2);
      sy = __fma_rn(x, y[i], sy);
      if (Xh) {
        const float h = __double2float_rn(x);
        Xh[(long long)j * ldh + i] = h;
        Xl[(long long)j * ldh + i] = __double2float_rn(__dsub_rn(x, (double)h));
      }
    }
    if (Xh)
      for (int i = n + lane; i < ldh; i += 32) {
        Xh[(long long)j * ldh + i] = 0.f;
        Xl[(long long)j * ldh + i] = 0.f;
      }
    s2 = warp_sum_d(s2);
    sy = warp_sum_d(sy);
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      if (!finite || !isfinite(sy)) atomicExch(&ctl->nonfinite, 1);
      const double nr = __dsqrt_rn(s2);
      nrm[j] = nr;
      nrmf[j] = __double2float_ru(nr);
      cy[j] = sy;
      const df2 iv = df_from_double(s2 > 0.0 ? __drcp_rn(s2) : 0.0);
      ftab[j] = make_float4(iv.h, iv.l, 0.f, 0.f);
      if (isfinite(sy)) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(fabs(sy)));
      const df2 bd = df_from_double(beta0 ? beta0[j] : 0.0);
      bdf[j] = make_float2(bd.h, bd.l);
      b0df[j] = make_float2(bd.h, bd.l);
    }
  }
}

// rho = y - X beta0 (FP64 per row), ||y||^2, eps = tol ||y||^2
template <typename XT>
__global__ void rho_init_kernel(const XT* X, long long ldx, int n, int p, const double* y, const double* beta0,
                                float* rho_h, float* rho_l, float* rho0_h, float* rho0_l, int ldh, double tol,
                                Ctrl* ctl) {
  __shared__ double buf[32];
  for (int i = blockIdx.x; i < ldh; i += gridDim.x) {
    double acc = 0.0;
    if (beta0 && i < n)
      for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const double b = beta0[j];
        if (b != 0.0) acc = __fma_rn(b, (double)X[(long long)j * ldx + i], acc);
      }
    acc = block_sum_d(acc, buf);
    if (threadIdx.x == 0) {
      const double r = (i < n) ? __dsub_rn(y[i], acc) : 0.0;
      if (!isfinite(r)) atomicExch(&ctl->nonfinite, 1);
      const df2 d = df_from_double(r);
      rho_h[i] = d.h;
      rho_l[i] = d.l;
      rho0_h[i] = d.h;
      rho0_l[i] = d.l;
    }
  }
  if (blockIdx.x == 0) {
    double yy = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) yy = __fma_rn(y[i], y[i], yy);
    yy = block_sum_d(yy, buf);
    if (threadIdx.x == 0) {
      ctl->yy = yy;
      ctl->eps = tol * yy;
    }
  }
}

// lambda_max = ||X^T y||_inf must be > 0 (otherwise every lambda_t is 0) and
// every ratio must lie in (0, 1]; violations are reported as INVALID_ARG.
// For the Elastic-Net with mixing a, beta = 0 is optimal from ||X^T y||_inf / a.
__global__ void finish_setup_kernel(Ctrl* ctl, const double* ratios, int T, double enet_alpha) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->lambda_max = __ddiv_rn(__longlong_as_double((long long)ctl->m_bits), enet_alpha);
    ctl->m_bits = 0ull;
    ctl->mlo_bits = 0u;
    bool bad = !(ctl->lambda_max > 0.0);
    for (int t = 0; t < T; ++t) bad = bad || !(ratios[t] > 0.0 && ratios[t] <= 1.0);
    if (ctl->nonfinite) ctl->err = kErrNonfinite;
    else if (bad) ctl->err = kErrInvalidArg;
  }
}

// stamp a device error into every stats record (after the path kernel)
__global__ void stats_error_kernel(Ctrl* ctl, lasso_path_stats* stats, int T) {
  const int e = ctl->err;
  if (e == 0) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    stats[t].status = e;
    stats[t].converged = 0;
  }
}

// ---------------------------------------------------------------- split-BF16 operands
// A value v (FP32) is carried as vh = bf16(v) and vl = bf16(v - vh), so that
// |v - vh - vl| <= 2^-16 |v|.  The three products that matter,
//   x.r ~ xh.rh + xh.rl + xl.rh   (the dropped xl.rl is <= 2^-16 |x r|),
// are one GEMM over a K dimension of 3 L: the design row j is packed as
// [xh | xh | xl] and the residual of problem b as [rh | rl | rh] (L = n
// rounded up to 8, zero padded).  Every product of two BF16 values is exact
// in FP32, so the error of c~ is at most (3 2^-16 + 2^-20) |x||r| plus the
// FP32 accumulation of 3 L terms.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
}

__global__ void pack_x_kernel(const float* __restrict__ X, long long ldx, int n, int p, int L,
                              __nv_bfloat16* __restrict__ X3) {
  const long long total = (long long)p * L;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / L), i = (int)(k % L);
    const float v = i < n ? X[(long long)j * ldx + i] : 0.f;
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* row = X3 + (long long)j * 3 * L;
    row[i] = h;
    row[L + i] = h;
    row[2 * L + i] = l;
  }
}

// residuals of the B problems: from the masked responses (first lambda) or
// from the FP32 high planes of the residuals kept in each problem's region
__global__ void pack_r_kernel(const double* Y, long long ldy, const uint8_t* rmask, long long ldm, const char* ws,
                              size_t region, size_t o_rho, int n, int B, int L, int from_y,
                              __nv_bfloat16* __restrict__ R3) {
  const long long total = (long long)B * L;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(k / L), i = (int)(k % L);
    float v = 0.f;
    if (i < n) {
      if (from_y) {
        const bool in = rmask == nullptr || rmask[i + (size_t)b * ldm] != 0;
        v = in ? (float)Y[i + (size_t)b * ldy] : 0.f;
      } else {
        v = reinterpret_cast<const float*>(ws + (size_t)b * region + o_rho)[i];
      }
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* row = R3 + (long long)b * 3 * L;
    row[i] = h;
    row[L + i] = l;
    row[2 * L + i] = h;
  }
}

// ---------------------------------------------------------------- host side
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxGrid = 1024;
constexpr int kSCapPath = 4096;   // chain entries per round, single path
constexpr int kSCapBatch = 512;   // chain entries per round, batched (per-CTA snapshots)

// Offsets of one workspace region (the single path has one; the batched
// solver one per resident CTA).  Planes of an FP64 design follow the region.
struct Layout {
  size_t o[32];
  size_t region, planes, total;
  long long ldw;
  int s_cap;
};
enum {
  L_ctrl, L_cnt, L_part_l1, L_nrm, L_nrmf, L_ftab, L_bdf, L_b0df, L_rho_h, L_rho_l, L_rho0_h, L_rho0_l, L_ctil,
  L_mask, L_A, L_sup0, L_sup1, L_chain, L_entered, L_oldb, L_recs, L_snap, L_zl_j, L_zl_b, L_zbits, L_yb, L_sk,
  L_mref, L_msnap, L_cy, L_part_l2, L_N
};

Layout make_layout(int64_t n, int64_t p, int s_cap_max, bool planes) {
  Layout L{};
  const long long ldw = (n + 3) / 4 * 4;
  const int s_cap = (int)std::min<int64_t>(s_cap_max, p);
  const int64_t words = (p + 31) / 32;
  size_t off = 0;
  auto take = [&](int k, size_t bytes) {
    L.o[k] = off;
    off += align256(bytes);
  };
  take(L_ctrl, sizeof(Ctrl));
  take(L_cnt, sizeof(int) * 4 * kMaxGrid);
  take(L_part_l1, sizeof(double) * kMaxGrid);
  take(L_nrm, sizeof(double) * p);
  take(L_nrmf, sizeof(float) * p);
  take(L_ftab, sizeof(float4) * p);
  take(L_bdf, sizeof(float2) * p);
  take(L_b0df, sizeof(float2) * p);
  take(L_rho_h, sizeof(float) * ldw);
  take(L_rho_l, sizeof(float) * ldw);
  take(L_rho0_h, sizeof(float) * ldw);
  take(L_rho0_l, sizeof(float) * ldw);
  take(L_ctil, sizeof(float) * p);
  take(L_mask, sizeof(uint32_t) * words);
  take(L_A, sizeof(int) * p);
  take(L_sup0, sizeof(int) * p);
  take(L_sup1, sizeof(int) * p);
  take(L_chain, sizeof(int) * (s_cap + 1));
  take(L_entered, sizeof(int) * p);
  take(L_oldb, sizeof(float2) * (s_cap + 1));
  take(L_recs, sizeof(ChainRec) * (s_cap + 1));
  take(L_snap, sizeof(float) * 2 * (size_t)ldw * (size_t)(s_cap + 2));
  take(L_zl_j, sizeof(int) * p);
  take(L_zl_b, sizeof(double) * p);
  take(L_zbits, sizeof(uint32_t) * words);
  take(L_yb, sizeof(double) * ldw);
  take(L_sk, sizeof(float) * p);
  take(L_mref, sizeof(float) * p);
  take(L_msnap, sizeof(float) * (s_cap + 2));
  take(L_cy, sizeof(double) * p);
  take(L_part_l2, sizeof(double) * kMaxGrid);
  L.region = off;
  L.planes = planes ? 2 * align256(sizeof(float) * (size_t)ldw * (size_t)p) : 0;
  L.total = L.region + L.planes;
  L.ldw = ldw;
  L.s_cap = s_cap;
  return L;
}

void set_offsets(Args& a, const Layout& L) {
  a.o_ctrl = L.o[L_ctrl];
  a.o_cnt_kept = L.o[L_cnt];
  a.o_cnt_sup = L.o[L_cnt] + sizeof(int) * kMaxGrid;
  a.o_cnt_nnz = L.o[L_cnt] + 2 * sizeof(int) * kMaxGrid;
  a.o_cnt_zero = L.o[L_cnt] + 3 * sizeof(int) * kMaxGrid;
  a.o_part_l1 = L.o[L_part_l1];
  a.o_nrm = L.o[L_nrm];
  a.o_nrmf = L.o[L_nrmf];
  a.o_ftab = L.o[L_ftab];
  a.o_bdf = L.o[L_bdf];
  a.o_b0df = L.o[L_b0df];
  a.o_rho_h = L.o[L_rho_h];
  a.o_rho_l = L.o[L_rho_l];
  a.o_rho0_h = L.o[L_rho0_h];
  a.o_rho0_l = L.o[L_rho0_l];
  a.o_ctil = L.o[L_ctil];
  a.o_mask = L.o[L_mask];
  a.o_A = L.o[L_A];
  a.o_sup0 = L.o[L_sup0];
  a.o_sup1 = L.o[L_sup1];
  a.o_chain = L.o[L_chain];
  a.o_entered = L.o[L_entered];
  a.o_oldb = L.o[L_oldb];
  a.o_recs = L.o[L_recs];
  a.o_snap = L.o[L_snap];
  a.o_zl_j = L.o[L_zl_j];
  a.o_zl_b = L.o[L_zl_b];
  a.o_zbits = L.o[L_zbits];
  a.o_yb = L.o[L_yb];
  a.o_sk = L.o[L_sk];
  a.o_mref = L.o[L_mref];
  a.o_msnap = L.o[L_msnap];
  a.o_cy = L.o[L_cy];
  a.o_part_l2 = L.o[L_part_l2];
  a.ldw = L.ldw;
  a.s_cap = L.s_cap;
}

template <int NGC, int CW, bool XLO, bool BATCH, int MINB = 1, bool EN = false>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&path_kernel<NGC, CW, XLO, BATCH, MINB, EN>);
}

// Chain shape for n rows.  A coordinate step is one warp's dependent
// instruction stream, so the chain spreads the rows until every lane holds a
// single float4 granule: one warp (no barrier, no shared-memory exchange)
// while n <= 128, four warps and 1, 2 or 4 granules per lane above.  Measured
// on the 500-row path: one warp with four granules per lane was 1.57x slower
// than four warps with one.
struct ChainShape {
  int cw, ngc;
};

ChainShape chain_shape(int64_t n, bool batch) {
  const int ld4 = (int)((n + 3) / 4);
  if (!batch && ld4 <= 32) return ChainShape{1, 1};
  return ChainShape{4, ld4 <= 128 ? 1 : (ld4 <= 256 ? 2 : 4)};
}

const void* pick_kernel(ChainShape c, bool xlo, bool batch, int per_sm = 1) {
  if (batch && per_sm == 2) return c.ngc == 1 ? kernel_ptr<1, 4, false, true, 2>()
                                 : c.ngc == 2 ? kernel_ptr<2, 4, false, true, 2>() : kernel_ptr<4, 4, false, true, 2>();
  if (batch) return c.ngc == 1 ? kernel_ptr<1, 4, false, true, 1>()
                  : c.ngc == 2 ? kernel_ptr<2, 4, false, true, 1>() : kernel_ptr<4, 4, false, true, 1>();
  if (c.cw == 1) return xlo ? kernel_ptr<1, 1, true, false>() : kernel_ptr<1, 1, false, false>();
  if (xlo) return c.ngc == 1 ? kernel_ptr<1, 4, true, false>()
                  : c.ngc == 2 ? kernel_ptr<2, 4, true, false>() : kernel_ptr<4, 4, true, false>();
  return c.ngc == 1 ? kernel_ptr<1, 4, false, false>()
         : c.ngc == 2 ? kernel_ptr<2, 4, false, false>() : kernel_ptr<4, 4, false, false>();
}

// the single path on an FP32 design with the Elastic-Net's ridge term
const void* pick_kernel_enet(ChainShape c) {
  if (c.cw == 1) return kernel_ptr<1, 1, false, false, 1, true>();
  return c.ngc == 1 ? kernel_ptr<1, 4, false, false, 1, true>()
         : c.ngc == 2 ? kernel_ptr<2, 4, false, false, 1, true>() : kernel_ptr<4, 4, false, false, 1, true>();
}

void fill_common(Args& a, int64_t n, int64_t p, int32_t T, const lasso_opts& o) {
  a.n = (int)n;
  a.p = (int)p;
  a.ld4 = (int)((n + 3) / 4);
  a.T = T;
  a.words = (int)((p + 31) / 32);
  a.f = o.screen_period;
  a.dual_point = o.dual_point;
  a.screen_rule = o.screen_rule;
  a.refined_radius = o.refined_radius;
  a.enet_alpha = o.enet_alpha;
  a.xtr_scope = o.xtr_scope;
  a.warm_start = o.warm_start;
  a.max_epochs = o.max_epochs;
  a.tol = o.gap_tol_rel;
}

// dynamic shared memory of a CTA: the feature list of a round and the ring
// of kRing staged columns (each chain thread's granules, two planes for FP64)
size_t dyn_smem(int s_cap, ChainShape c, bool xlo) {
  const size_t jl_bytes = (((size_t)(s_cap + 1) * sizeof(int)) + 127) & ~(size_t)127;
  return jl_bytes + (size_t)kRing * c.ngc * 32 * c.cw * 16 * (xlo ? 2 : 1);
}

struct DevInfo {
  int sms, coop, smem_optin;
};

lasso_status dev_info(DevInfo& d) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.coop, cudaDevAttrCooperativeLaunch, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return LASSO_OK;
}

// resident CTAs of the batched solver for a given device (fixed, so that the
// workspace size does not depend on the occupancy query)
int batch_grid(int64_t B, int sms, int per_sm = 2) {
  return (int)std::min<int64_t>(B, std::min<int64_t>((int64_t)sms * per_sm, kMaxGrid));
}

}  // namespace

size_t path_workspace_size(int64_t n, int64_t p, lasso_dtype xt, int64_t ldx) {
  (void)ldx;
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4) return 0;
  if (xt != LASSO_F32 && xt != LASSO_F64) return 0;
  return make_layout(n, p, kSCapPath, xt == LASSO_F64).total;
}

lasso_status path_launch(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx, const double* y,
                         const double* ratios, int32_t T, const double* beta0, const lasso_opts& o,
                         double* beta_out, uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                         cudaStream_t stream) {
  const bool f64 = xt == LASSO_F64;
  const Layout L = make_layout(n, p, kSCapPath, f64);
  if (ws_bytes < L.total)
    return set_error(LASSO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes required", ws_bytes,
                     L.total);
  char* base = static_cast<char*>(ws);
  Args a{};
  fill_common(a, n, p, T, o);
  set_offsets(a, L);
  a.ws = base;
  a.cta_bytes = 0;
  a.B = 1;
  a.y = y;
  a.ratios = ratios;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  float* Xh_w = reinterpret_cast<float*>(base + L.region);
  float* Xl_w = reinterpret_cast<float*>(base + L.region + L.planes / 2);
  if (f64) {
    a.Xh = Xh_w;
    a.Xl = Xl_w;
    a.ldx = L.ldw;
  } else {
    a.Xh = static_cast<const float*>(X);
    a.Xl = nullptr;
    a.ldx = ldx;
  }
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + a.o_ctrl);
  const ChainShape cs = chain_shape(n, false);
  const bool enet = o.enet_alpha < 1.0;
  if (enet && f64) return set_error(LASSO_ERR_INVALID_ARG, "enet_alpha < 1 needs an FP32 design");
  const void* kfn = enet ? pick_kernel_enet(cs) : pick_kernel(cs, f64, false);
  DevInfo d{};
  lasso_status st = dev_info(d);
  if (st != LASSO_OK) return st;
  if (!d.coop) return set_error(LASSO_ERR_CUDA, "device does not support cooperative launch");
  const size_t dyn = dyn_smem(L.s_cap, cs, f64);
  if (dyn + 8192 > (size_t)d.smem_optin)
    return set_error(LASSO_ERR_INVALID_ARG, "the chain ring of %zu bytes does not fit shared memory", dyn);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, dyn));
  if (per_sm < 1) return set_error(LASSO_ERR_CUDA, "the path kernel cannot be resident (occupancy 0)");
  per_sm = std::min(per_sm, 2);
  const int grid = std::min(d.sms * per_sm, kMaxGrid);
  const int fs = (int)((p + grid - 1) / grid);
  a.fs = (fs + 31) / 32 * 32;

  CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream));
  CUDA_TRY(cudaMemsetAsync(base + a.o_cnt_kept, 0, sizeof(int) * 4 * kMaxGrid, stream));
  double* nrm = reinterpret_cast<double*>(base + a.o_nrm);
  float* nrmf = reinterpret_cast<float*>(base + a.o_nrmf);
  float4* ftab = reinterpret_cast<float4*>(base + a.o_ftab);
  float2* bdf = reinterpret_cast<float2*>(base + a.o_bdf);
  float2* b0df = reinterpret_cast<float2*>(base + a.o_b0df);
  double* cy = reinterpret_cast<double*>(base + a.o_cy);
  float* rho_h = reinterpret_cast<float*>(base + a.o_rho_h);
  float* rho_l = reinterpret_cast<float*>(base + a.o_rho_l);
  float* rho0_h = reinterpret_cast<float*>(base + a.o_rho0_h);
  float* rho0_l = reinterpret_cast<float*>(base + a.o_rho0_l);
  const int blocks = d.sms * 8;
  if (f64)
    precompute_kernel<double><<<blocks, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                          Xh_w, Xl_w, a.ldw, nrm, nrmf, ftab, bdf, b0df, cy, ctrl);
  else
    precompute_kernel<float><<<blocks, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                         nullptr, nullptr, a.ldw, nrm, nrmf, ftab, bdf, b0df, cy, ctrl);
  CUDA_TRY(cudaGetLastError());
  const int rb = (int)std::min<long long>(a.ldw, (long long)d.sms * 4);
  if (f64)
    rho_init_kernel<double><<<rb, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                    rho_h, rho_l, rho0_h, rho0_l, (int)a.ldw, o.gap_tol_rel, ctrl);
  else
    rho_init_kernel<float><<<rb, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                   rho_h, rho_l, rho0_h, rho0_l, (int)a.ldw, o.gap_tol_rel, ctrl);
  CUDA_TRY(cudaGetLastError());
  finish_setup_kernel<<<1, 32, 0, stream>>>(ctrl, ratios, T, o.enet_alpha);
  CUDA_TRY(cudaGetLastError());
  void* params[] = {&a};
  CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
  stats_error_kernel<<<1, 128, 0, stream>>>(ctrl, stats, T);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

// ---------------------------------------------------------------- batched
namespace {
struct BatchLayout {
  Layout L;
  int grid, regions;
  bool lockstep;
  long long Lk;  // K segment length of the split-BF16 operands
  size_t o_regions, o_x3, o_r3, o_c, o_gerr, total;
};

BatchLayout batch_layout(int64_t n, int64_t p, int64_t B, bool lockstep, int sms) {
  BatchLayout bl{};
  bl.L = make_layout(n, p, kSCapBatch, false);
  bl.grid = batch_grid(B, sms);
  bl.lockstep = lockstep;
  bl.regions = lockstep ? (int)B : bl.grid;
  bl.Lk = (n + 7) / 8 * 8;
  size_t off = 256;
  bl.o_regions = off;
  off += bl.L.region * (size_t)bl.regions;
  if (lockstep) {
    bl.o_x3 = off;
    off += align256(sizeof(__nv_bfloat16) * 3 * (size_t)bl.Lk * (size_t)p);
    bl.o_r3 = off;
    off += align256(sizeof(__nv_bfloat16) * 3 * (size_t)bl.Lk * (size_t)B);
    bl.o_c = off;
    off += align256(sizeof(float) * (size_t)p * (size_t)B);
    bl.o_gerr = off;
    off += 256;
  }
  bl.total = off;
  return bl;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  return sms;
}
}  // namespace

size_t batch_workspace_size(int64_t n, int64_t p, int64_t B, bool lockstep) {
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4 || B < 1) return 0;
  return batch_layout(n, p, B, lockstep, device_sms()).total;
}

lasso_status batch_launch(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                          const uint8_t* row_mask, int64_t ldm, int64_t B, const double* ratios, int32_t T,
                          const double* beta0, int64_t ldb0, const lasso_opts& o, double* beta_out,
                          uint32_t* mask_out, lasso_path_stats* stats,
                          void* ws, size_t ws_bytes, cudaStream_t stream) {
  DevInfo d{};
  lasso_status st = dev_info(d);
  if (st != LASSO_OK) return st;
  const bool lockstep = o.gemm_dtype == LASSO_BF16;
  const BatchLayout bl = batch_layout(n, p, B, lockstep, d.sms);
  if (ws_bytes < bl.total)
    return set_error(LASSO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes required", ws_bytes,
                     bl.total);
  char* base = static_cast<char*>(ws);
  Args a{};
  fill_common(a, n, p, T, o);
  set_offsets(a, bl.L);
  a.ws = base + bl.o_regions;
  a.cta_bytes = bl.L.region;
  a.B = (int)B;
  a.y = Y;
  a.ldy = ldy;
  a.rmask = row_mask;
  a.ldm = ldm;
  a.beta0 = beta0;
  a.ldb0 = ldb0;
  a.queue = reinterpret_cast<int*>(base);
  a.ratios = ratios;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  a.Xh = X;
  a.Xl = nullptr;
  a.ldx = ldx;
  a.fs = (int)((p + 31) / 32 * 32);
  a.gsize = 1;
  const ChainShape cs = chain_shape(n, true);
  const int per_sm = o.batch_ctas_per_sm == 1 ? 1 : 2;
  const int grid = batch_grid(B, d.sms, per_sm);  // <= the regions the layout holds
  const void* kfn = pick_kernel(cs, false, true, per_sm);
  const size_t dyn = dyn_smem(bl.L.s_cap, cs, false);
  if (dyn + 8192 > (size_t)d.smem_optin)
    return set_error(LASSO_ERR_INVALID_ARG, "the chain ring of %zu bytes does not fit shared memory", dyn);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  if (!lockstep && o.batch_group > 1) {
    // groups of CTAs per problem: every group's CTAs must be resident together
    // (their barrier), so the launch is cooperative and fills the resident CTAs
    const int gs = o.batch_group;
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kThreads, dyn));
    const int resident = d.sms * std::min(occ, per_sm);
    const int groups = (int)std::min<int64_t>(B, resident / gs);
    if (groups < 1)
      return set_error(LASSO_ERR_INVALID_ARG, "batch_group %d exceeds the %d resident CTAs", gs, resident);
    a.gsize = gs;
    const long long fsz = (p + gs - 1) / gs;
    a.fs = (int)((fsz + 31) / 32 * 32);
    // each group's control block (its barrier count) starts at zero
    CUDA_TRY(cudaMemset2DAsync(a.ws + a.o_ctrl, a.cta_bytes, 0, sizeof(Ctrl), (size_t)groups, stream));
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(groups * gs), dim3(kThreads), params, dyn, stream));
    return LASSO_OK;
  }
  if (!lockstep) {
    // each CTA solves whole paths; its first checks are CUDA-core FP32 passes
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
    return LASSO_OK;
  }
  // lockstep: per lambda, the residuals of all problems -> one tensor-core
  // product C = X^T R (split BF16) -> one launch that advances every problem
  // by one lambda, its first check reading C with the split-BF16 error factor
  const long long Lk = bl.Lk;
  __nv_bfloat16* X3 = reinterpret_cast<__nv_bfloat16*>(base + bl.o_x3);
  __nv_bfloat16* R3 = reinterpret_cast<__nv_bfloat16*>(base + bl.o_r3);
  float* C = reinterpret_cast<float*>(base + bl.o_c);
  int* gerr = reinterpret_cast<int*>(base + bl.o_gerr);
  a.lockstep = 1;
  a.cfirst = C;
  a.ldc = p;
  a.cfactor = (float)((3.0 * 0x1p-16 + 0x1p-20 + (3.0 * (double)Lk + 8.0) * 0x1p-24) * 1.05);
  CUDA_TRY(cudaMemsetAsync(gerr, 0, 256, stream));
  pack_x_kernel<<<d.sms * 8, 256, 0, stream>>>(X, ldx, (int)n, (int)p, (int)Lk, X3);
  CUDA_TRY(cudaGetLastError());
  for (int t = 0; t < T; ++t) {
    // the product must be taken on the residual the lambda starts from: y at
    // t = 0 (zero start), rho0 = y - X beta0 when every lambda restarts, else
    // the previous lambda's final residual.  At t = 0 with beta0 the residual
    // is formed inside the launch, so that first check runs the FP32 pass.
    const bool use_gemm = !(t == 0 && beta0 != nullptr);
    if (use_gemm) {
      pack_r_kernel<<<d.sms * 4, 256, 0, stream>>>(Y, ldy, row_mask, ldm, a.ws, a.cta_bytes,
                                                   o.warm_start ? a.o_rho_h : a.o_rho0_h, (int)n, (int)B, (int)Lk,
                                                   t == 0 ? 1 : 0, R3);
      CUDA_TRY(cudaGetLastError());
      st = xtr_gemm_launch(X3, 3 * Lk, p, 3 * Lk, R3, 3 * Lk, B, C, p, gerr, stream, o.gemm_tile_n);
      if (st != LASSO_OK) return st;
    }
    a.cfirst = use_gemm ? C : nullptr;
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    a.t0 = t;
    a.t1 = t + 1;
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
  }
  return LASSO_OK;
}

}  // namespace lassogs
