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
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "cd_common.cuh"
#include "gram_chain.cuh"
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
  // Gram rounds in detail: [0] chain warp waiting for its helpers, [1] chain
  // warp busy, [2] helper warp 1 busy, [3] publisher busy, [4] snapshot CTA 1
  // waiting for published entries, [5] snapshot CTA 1 busy, [6] Gram rounds,
  // [7] direct rounds.  One-CTA problems instead: [0] rounds, [1] positions
  // scanned by the verification, [2] columns it read, [3] its exact
  // refinements, [4] cycles of the snapshot distances
  unsigned long long gprof[8];
  int win;                    // positions a round may span (adaptive, see the passes)
  int prob;                   // groups of CTAs: the problem CTA 0 took from the queue
  // Gram form of the chain (single path): slots of the lambda's cache, whether
  // it is in use, the form of the planned round (0 direct, 1 Gram), the slot
  // an entering feature gets in it (-1 none) and the entries of the round
  // whose updates are published
  int nslots, gram_on, rmode, newslot, pub_g;
  // lockstep batches advancing one pass per launch: the lambda index, whether
  // the next launch resumes inside it, the next pass of the period, the
  // support list in use (0: sup0, 1: sup1), the lambda's counters so far, and
  // whether the path is finished
  int t_cur, resume, e_cur, sup_par, pdone, scope_s;
  float anorm;                // bound on ||anchor|| (one-CTA problems)
  long long ep_s, ck_s, xc_s;
  // audit of the correlation bounds: largest |c~ - c| / E of the lambda so
  // far (FP64 bits), for CUDA-core and tensor-core correlations
  unsigned long long aud_bits, aud_tc_bits;
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
  int audit;        // 1: record |c~ - c| / E at every check (lasso_opts.audit_bounds)
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
  // pass_mode: each launch advances every problem by one pass (after the
  // checks that are due), every check and the certificates of every pass
  // come from cfirst, and t0 = 0 marks the first launch; active counts the
  // problems whose path is not finished
  int pass_mode;
  int* active;
  // park: a problem that finishes a lambda stops there and records the next
  // lambda in park_t[b] (the host solves the rest of its path on the single
  // path); set for the last few unfinished problems of a batch without row subsets
  int park;
  int* park_t;
  const float* cfirst;
  long long ldc;
  float cfactor;
  unsigned long long wait_ns;  // time limit of every grid-barrier wait
  // Gram form of the chain (single path; gram_cap = 0 switches it off):
  // G = X_S^T X_S over the cache slots (gram_cap x gram_cap double-floats),
  // slot of a feature, feature of a slot, x_c^T rho_0 per chain entry, the
  // published update of each entry; nsc CTAs (1..nsc) rebuild the snapshots
  size_t o_gram, o_slot, o_feat, o_g0, o_dlt;
  // one-CTA problems: the residual the certificates were last issued from
  // (the anchor, high plane), the distance of each snapshot of a round from
  // it, and the distance of the residual each certificate was issued at
  size_t o_anchor, o_dsnap, o_dref;
  int gram_cap, nsc;
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
      ctl->aud_bits = 0ull;
      ctl->aud_tc_bits = 0ull;
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
      // the Elastic-Net with mixing a: beta = 0 is optimal from ||X^T y||_inf / a
      ctl->lambda_max = __ddiv_rn(__longlong_as_double((long long)ctl->m_bits), a.enet_alpha);
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

// ---------------------------------------------------------------- Gram rounds
// Shared memory of a Gram round of CTA 0 (dynamic shared memory, used only
// while the round runs): per chain entry its feature, cache slot, the
// coordinate table, beta before the round, ||x_j|| rounded up, x_c^T rho_0,
// the update and the new coefficient; per block of 32 entries (two buffers)
// the helpers' partial corrections and the two 32 x 32 tiles of G the chain
// warp uses.
struct GramSmem {
  float4* tab;
  float2 *b, *gz, *d, *nb, *part, *Gd, *Go;
  int *j, *sl;
  float* nf;
};
constexpr size_t kGramSmemBytes = (size_t)kGramMaxNc * (16 + 8 + 8 + 8 + 8 + 4 + 4 + 4) +
                                  sizeof(float2) * (2 * kGramHelpers * 32 + 2 * 2 * 32 * 32);

__device__ __forceinline__ GramSmem gram_smem(unsigned char* base) {
  GramSmem g;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += bytes;
    return p;
  };
  g.tab = reinterpret_cast<float4*>(take(16 * (size_t)kGramMaxNc));
  g.b = reinterpret_cast<float2*>(take(8 * (size_t)kGramMaxNc));
  g.gz = reinterpret_cast<float2*>(take(8 * (size_t)kGramMaxNc));
  g.d = reinterpret_cast<float2*>(take(8 * (size_t)kGramMaxNc));
  g.nb = reinterpret_cast<float2*>(take(8 * (size_t)kGramMaxNc));
  g.part = reinterpret_cast<float2*>(take(sizeof(float2) * 2 * kGramHelpers * 32));
  g.Gd = reinterpret_cast<float2*>(take(sizeof(float2) * 2 * 32 * 32));
  g.Go = reinterpret_cast<float2*>(take(sizeof(float2) * 2 * 32 * 32));
  g.j = reinterpret_cast<int*>(take(4 * (size_t)kGramMaxNc));
  g.sl = reinterpret_cast<int*>(take(4 * (size_t)kGramMaxNc));
  g.nf = reinterpret_cast<float*>(take(4 * (size_t)kGramMaxNc));
  return g;
}

// One round of the coordinate chain in Gram form, run by the whole of CTA 0.
// Entry c of the chain has g_c = x_c^T rho_0 - sum_{c' < c} delta_c' G[c][c']
// (x_c^T rho_0 from the prep phase, in g0).  The entries are taken in blocks
// of 32, one per lane of warp 0:
//   warp 0 (chain)   per block: g minus the helpers' corrections (blocks up to
//                    two back), minus the block before through its deltas,
//                    then 32 sequential soft-threshold steps; after step i
//                    the delta of lane i is broadcast and every later lane
//                    subtracts delta_i G[c][c_i].
//   warps 1-3, 5-7   (helpers) per block T: the partial sums
//                    sum delta_c' G[c][c'] over the blocks up to T - 2 (rows
//                    split over the helpers), and the tiles G(T, T), G(T-1, T)
//                    staged in shared memory.
//   warp 4           (publisher) per finished block: new coefficients, old
//                    ones and deltas to global memory, the movement counter,
//                    then the count of published entries that the snapshot
//                    CTAs follow.
// Every wait is a bounded spin on a shared-memory counter; on expiry the round
// unwinds and LASSO_ERR_TIMEOUT is recorded.
template <int NG, bool XLO, bool EN>
__device__ void gram_round(const Args& a, char* wsb, Ctrl* ctl, unsigned char* dsm, volatile int* gf, int nc,
                           int newslot, df2 ridge, int* err) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned FULL = 0xffffffffu;
  GramSmem S = gram_smem(dsm);
  const int cap = a.gram_cap;
  const float2* Gm = reinterpret_cast<const float2*>(wsb + a.o_gram);
  const int* chain = reinterpret_cast<const int*>(wsb + a.o_chain);
  const int* A = reinterpret_cast<const int*>(wsb + a.o_A);
  int* slot = reinterpret_cast<int*>(wsb + a.o_slot);
  int* feat = reinterpret_cast<int*>(wsb + a.o_feat);
  const float2* g0 = reinterpret_cast<const float2*>(wsb + a.o_g0);
  const float4* ftab = reinterpret_cast<const float4*>(wsb + a.o_ftab);
  float2* bdf = reinterpret_cast<float2*>(wsb + a.o_bdf);
  const float* nrmf = reinterpret_cast<const float*>(wsb + a.o_nrmf);
  float2* oldb = reinterpret_cast<float2*>(wsb + a.o_oldb);
  float2* dlt = reinterpret_cast<float2*>(wsb + a.o_dlt);
  float* msnap = reinterpret_cast<float*>(wsb + a.o_msnap);
  // the entering feature (chain entry 0) takes its slot in the cache
  if (tid == 0 && newslot >= 0) {
    const int jf = __ldcg(A + __ldcg(chain));
    slot[jf] = newslot;
    feat[newslot] = jf;
    ctl->nslots = newslot + 1;
  }
  for (int c = tid; c < nc; c += kThreads) {
    const int j = __ldcg(A + __ldcg(chain + c));
    S.j[c] = j;
    S.sl[c] = (c == 0 && newslot >= 0) ? newslot : __ldcg(slot + j);
    S.tab[c] = __ldcg(ftab + j);
    S.b[c] = __ldcg(bdf + j);
    S.nf[c] = __ldcg(nrmf + j);
    S.gz[c] = __ldcg(g0 + c);
  }
  if (tid < 16) gf[tid] = 0;  // [0] blocks done by the chain warp, [1] abort, [2..8) helper progress
  __syncthreads();
  const int nblk = (nc + 31) >> 5;
  if (warp == 0) {
    // ---- the chain.  Lane l carries the unthresholded update of its
    // coordinate, u_l = beta_l + g_l / ||x_l||^2 (the Elastic-Net's ridge term
    // folded in); a step of coordinate i is nb_i = ST(u_i, thr_i), broadcast,
    // and u_l -= (nb_i - beta_i) G[i][l] / ||x_l||^2 for the later lanes.  The
    // tile Gd is staged already divided by ||x_l||^2.
    df2 dprev{0.f, 0.f};
    long long t_wait = 0, t_busy = 0, tc = clock64();
    for (int T = 0; T < nblk; ++T) {
      bool ok = true;
      for (int w = 0; w < kGramHelpers && ok; ++w) ok = smem_wait_ge(gf + 2 + w, T + 1, gf + 1, a.wait_ns, false);
      {
        const long long now = clock64();
        t_wait += now - tc;
        tc = now;
      }
      if (!__all_sync(FULL, ok)) break;
      __threadfence_block();
      const int c = 32 * T + lane;
      const bool valid = c < nc;
      const int cnt = min(32, nc - 32 * T);
      const int buf = T & 1;
      const float2* Gd = S.Gd + buf * 1024;
      const float2* Go = S.Go + buf * 1024;
      const float2* part = S.part + buf * kGramHelpers * 32;
      df2 g{0.f, 0.f}, beta{0.f, 0.f};
      float4 tb = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) {
        const float2 z = S.gz[c], bb = S.b[c];
        g = df2{z.x, z.y};
        beta = df2{bb.x, bb.y};
        tb = S.tab[c];
      }
      df2 acc{0.f, 0.f};
#pragma unroll
      for (int w = 0; w < kGramHelpers; ++w) {
        const float2 pz = part[w * 32 + lane];
        acc = df_add(acc, df2{pz.x, pz.y});
      }
      g = df_sub(g, acc);
      if (T > 0) {
        df2 a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
#pragma unroll 2
        for (int i = 0; i < 32; i += 4) {
          const float dh0 = __shfl_sync(FULL, dprev.h, i), dl0 = __shfl_sync(FULL, dprev.l, i);
          const float dh1 = __shfl_sync(FULL, dprev.h, i + 1), dl1 = __shfl_sync(FULL, dprev.l, i + 1);
          const float dh2 = __shfl_sync(FULL, dprev.h, i + 2), dl2 = __shfl_sync(FULL, dprev.l, i + 2);
          const float dh3 = __shfl_sync(FULL, dprev.h, i + 3), dl3 = __shfl_sync(FULL, dprev.l, i + 3);
          const float2 G0 = Go[i * 32 + lane], G1 = Go[(i + 1) * 32 + lane];
          const float2 G2 = Go[(i + 2) * 32 + lane], G3 = Go[(i + 3) * 32 + lane];
          a0 = df_sub_mul(a0, df2{-dh0, -dl0}, df2{G0.x, G0.y});
          a1 = df_sub_mul(a1, df2{-dh1, -dl1}, df2{G1.x, G1.y});
          a2 = df_sub_mul(a2, df2{-dh2, -dl2}, df2{G2.x, G2.y});
          a3 = df_sub_mul(a3, df2{-dh3, -dl3}, df2{G3.x, G3.y});
        }
        g = df_sub(g, df_add(df_add(a0, a1), df_add(a2, a3)));
      }
      // Elastic-Net: the augmented correlation is g - mu beta (beta_c changes
      // only at the entry's own step)
      if (EN) g = df_sub(g, df_mul(ridge, beta));
      const df2 thr{tb.z, tb.w};
      df2 u = df_add(beta, df_mul(g, df2{tb.x, tb.y}));
      df2 mynb = beta;
      if (cnt == 32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float2 Gi = Gd[i * 32 + lane];
          const float bh = __shfl_sync(FULL, beta.h, i), bl = __shfl_sync(FULL, beta.l, i);
          const df2 v = df_sub_mul(u, df2{-bh, -bl}, df2{Gi.x, Gi.y});
          const df2 nbv = soft_threshold_df(u, thr);
          const float nh = __shfl_sync(FULL, nbv.h, i), nl = __shfl_sync(FULL, nbv.l, i);
          if (lane == i) mynb = nbv;
          const df2 un = df_sub_mul(v, df2{nh, nl}, df2{Gi.x, Gi.y});
          u = lane > i ? un : u;
        }
      } else {
        for (int i = 0; i < cnt; ++i) {
          const float2 Gi = Gd[i * 32 + lane];
          const float bh = __shfl_sync(FULL, beta.h, i), bl = __shfl_sync(FULL, beta.l, i);
          const df2 v = df_sub_mul(u, df2{-bh, -bl}, df2{Gi.x, Gi.y});
          const df2 nbv = soft_threshold_df(u, thr);
          const float nh = __shfl_sync(FULL, nbv.h, i), nl = __shfl_sync(FULL, nbv.l, i);
          if (lane == i) mynb = nbv;
          const df2 un = df_sub_mul(v, df2{nh, nl}, df2{Gi.x, Gi.y});
          u = lane > i ? un : u;
        }
      }
      // the update of each coordinate: new minus old (exactly -beta when it
      // becomes zero, as nb = 0 then)
      const df2 myd = valid ? df_sub(mynb, beta) : df2{0.f, 0.f};
      if (valid) {
        S.d[c] = make_float2(myd.h, myd.l);
        S.nb[c] = make_float2(mynb.h, mynb.l);
      }
      dprev = myd;
      __syncwarp();
      __threadfence_block();
      if (lane == 0) gf[0] = T + 1;
      const long long now = clock64();
      t_busy += now - tc;
      tc = now;
    }
    if (lane == 0) {
      ctl->gprof[0] += (unsigned long long)t_wait;
      ctl->gprof[1] += (unsigned long long)t_busy;
      ctl->gprof[6] += 1ull;
    }
  } else if (warp == 4) {
    // ---- the publisher
    float run = __shfl_sync(FULL, lane == 0 ? __ldcg(msnap) : 0.f, 0);
    long long t_busy = 0;
    for (int m = 0; m < nblk; ++m) {
      const bool ok = smem_wait_ge(gf, m + 1, gf + 1, a.wait_ns, true);
      if (!__all_sync(FULL, ok)) break;
      const long long t0 = clock64();
      __threadfence_block();
      const int c = 32 * m + lane;
      const bool valid = c < nc;
      float mv = 0.f;
      if (valid) {
        const float2 dd = S.d[c];
        bdf[S.j[c]] = S.nb[c];
        oldb[c] = S.b[c];
        dlt[c] = dd;
        mv = __fmul_ru(__fadd_ru(fabsf(dd.x), fabsf(dd.y)), S.nf[c]);
      }
      // movement bound after each entry: an inclusive scan rounded up, so
      // every prefix bounds sum |delta_c| ||x_c||
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_up_sync(FULL, mv, o);
        if (lane >= o) mv = __fadd_ru(mv, u);
      }
      const float pre = __fadd_ru(run, mv);
      if (valid) msnap[c + 1] = pre;
      run = __shfl_sync(FULL, pre, 31);
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        *(volatile int*)&ctl->pub_g = min(32 * (m + 1), nc);
      }
      t_busy += clock64() - t0;
    }
    if (lane == 0) ctl->gprof[3] += (unsigned long long)t_busy;
  } else {
    // ---- helpers
    const int hw = warp < 4 ? warp - 1 : warp - 2;
    long long t_busy = 0;
    for (int T = 0; T < nblk; ++T) {
      const int buf = T & 1;
      if (T >= 2) {
        const bool ok = smem_wait_ge(gf, T - 1, gf + 1, a.wait_ns, true);
        if (!__all_sync(FULL, ok)) break;
        __threadfence_block();
      }
      const long long t0 = clock64();
      const int cl = 32 * T + lane;
      const bool vl = cl < nc;
      const size_t slc = vl ? (size_t)S.sl[cl] : 0;
      // partial sums over the entries r of the blocks up to T - 2 (rows of G
      // read at the columns of block T: one coalesced row segment per step)
      const int rows = 32 * (T - 1);
      constexpr int kB = 16;  // rows in flight per helper lane
      df2 acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = df2{0.f, 0.f};
      int r = hw;
      for (; r + (kB - 1) * kGramHelpers < rows; r += kB * kGramHelpers) {
        float2 Gv[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const int rr = r + u * kGramHelpers;
          Gv[u] = vl ? __ldcg(Gm + (size_t)S.sl[rr] * cap + slc) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const float2 dd = S.d[r + u * kGramHelpers];
          acc[u & 7] = df_sub_mul(acc[u & 7], df2{-dd.x, -dd.y}, df2{Gv[u].x, Gv[u].y});
        }
      }
      for (; r < rows; r += kGramHelpers) {
        const float2 Gv = vl ? __ldcg(Gm + (size_t)S.sl[r] * cap + slc) : make_float2(0.f, 0.f);
        const float2 dd = S.d[r];
        acc[0] = df_sub_mul(acc[0], df2{-dd.x, -dd.y}, df2{Gv.x, Gv.y});
      }
      df2 tot = acc[0];
#pragma unroll
      for (int u = 1; u < 8; ++u) tot = df_add(tot, acc[u]);
      S.part[buf * kGramHelpers * 32 + hw * 32 + lane] = make_float2(tot.h, tot.l);
      // tiles of block T: G(T, T) below the diagonal in the chain's order,
      // divided by ||x_l||^2 of the lane's coordinate, and G(T - 1, T)
      const float4 tl = vl ? S.tab[cl] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = hw; i < 32; i += kGramHelpers) {
        const int ci = 32 * T + i;
        float2 gd = make_float2(0.f, 0.f);
        if (vl && lane > i) {
          const float2 gv = __ldcg(Gm + (size_t)S.sl[ci] * cap + slc);
          const df2 sc = df_mul(df2{gv.x, gv.y}, df2{tl.x, tl.y});
          gd = make_float2(sc.h, sc.l);
        }
        S.Gd[buf * 1024 + i * 32 + lane] = gd;
        if (T > 0) {
          const int cp = 32 * (T - 1) + i;
          S.Go[buf * 1024 + i * 32 + lane] = vl ? __ldcg(Gm + (size_t)S.sl[cp] * cap + slc) : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      __threadfence_block();
      if (lane == 0) gf[2 + hw] = T + 1;
      t_busy += clock64() - t0;
    }
    if (hw == 0 && lane == 0) ctl->gprof[2] += (unsigned long long)t_busy;
  }
  __syncthreads();
  if (tid == 0 && gf[1] != 0) set_error(err, kErrTimeout);
}

// Residual snapshots of a Gram round, rebuilt from the published updates:
// snapshot c + 1 = snapshot c - delta_c x_c (the axpy of the direct chain, in
// the same double-float arithmetic).  CTA 1 + part runs rows
// [256 part, 256 part + 256) of the snapshot planes, the padding rows n..ldw-1
// included (they must stay as in snapshot 0, since a snapshot is later copied
// to the front whole): each of its first four warps owns 64 rows, two per
// lane.  The columns of a block of 32 entries are copied into a
// shared-memory ring (cp.async) while the block before is processed.  The
// waits for published entries are bounded and give up when another CTA has
// recorded an error.
constexpr int kFollowRows = 256;  // rows of one snapshot CTA
template <bool XLO>
__device__ void snapshot_follow(const Args& a, char* wsb, Ctrl* ctl, unsigned char* dsm, int nc, int part, int* err,
                                const uint8_t* rm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp >= 4) return;
  const unsigned FULL = 0xffffffffu;
  const int g2 = (kFollowRows / 2) * part + tid;  // float2 granule: rows 2 g2, 2 g2 + 1
  const int r0 = 2 * g2;
  const bool valid = r0 < a.ldw;  // ldw is a multiple of 4, so r0 + 1 < ldw too
  // rows of the design (x is 0 below them) and of the problem's row subset
  const bool in0 = r0 < a.n && (rm == nullptr || rm[r0] != 0);
  const bool in1 = r0 + 1 < a.n && (rm == nullptr || rm[r0 + 1] != 0);
  float* snap = reinterpret_cast<float*>(wsb + a.o_snap);
  const int* chain = reinterpret_cast<const int*>(wsb + a.o_chain);
  const int* A = reinterpret_cast<const int*>(wsb + a.o_A);
  const float2* dlt = reinterpret_cast<const float2*>(wsb + a.o_dlt);
  // ring[buf][entry][thread] (xh, then xl for an FP64 design)
  float2* ring = reinterpret_cast<float2*>(dsm);
  constexpr int kPl = XLO ? 2 : 1;
  auto slot_of = [&](int buf, int i, int pl) { return ring + (((buf * 32 + i) * kPl + pl) * 128 + tid); };
  float2 rh = valid ? __ldcg(reinterpret_cast<const float2*>(snap) + g2) : make_float2(0.f, 0.f);
  float2 rl = valid ? __ldcg(reinterpret_cast<const float2*>(snap + a.ldw) + g2) : make_float2(0.f, 0.f);
  const int nblk = (nc + 31) >> 5;
  auto stage = [&](int m) {
    if (m < nblk) {
      const int c = 32 * m + lane;
      const int jc = c < nc ? __ldcg(A + __ldcg(chain + c)) : 0;
      for (int i = 0; i < 32; ++i) {
        const int j = __shfl_sync(FULL, jc, i);
        if (valid && 32 * m + i < nc) {
          cp_async8(slot_of(m & 1, i, 0), a.Xh + (long long)j * a.ldx + r0);
          if (XLO) cp_async8(slot_of(m & 1, i, 1), a.Xl + (long long)j * a.ldx + r0);
        }
      }
    }
    cp_async_commit();
  };
  stage(0);
  for (int m = 0; m < nblk; ++m) {
    stage(m + 1);
    const int need = min(32 * (m + 1), nc);
    bool ok = true;
    const long long tw0 = clock64();
    if (lane == 0) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_volatile(&ctl->pub_g) < need) {
        __nanosleep(32);
        if ((++spins & 63u) == 0u) {
          if (ld_volatile(err) != 0) {
            ok = false;
            break;
          }
          if (global_ns() - t0 > a.wait_ns) {
            set_error(err, kErrTimeout);
            ok = false;
            break;
          }
        }
      }
    }
    if (!__shfl_sync(FULL, ok, 0)) {
      cp_async_wait<0>();
      return;
    }
    const long long tw1 = clock64();
    if (part == 0 && tid == 0) ctl->gprof[4] += (unsigned long long)(tw1 - tw0);
    __threadfence();
    cp_async_wait<1>();  // the columns of block m have landed
    __syncwarp();
    const int c = 32 * m + lane;
    const int cnt = min(32, nc - 32 * m);
    const float2 dl = c < nc ? __ldcg(dlt + c) : make_float2(0.f, 0.f);
    const int buf = m & 1;
    auto step = [&](int i, float2 xh, float2 xl) {
      const float dh = __shfl_sync(FULL, dl.x, i), dlo = __shfl_sync(FULL, dl.y, i);
      if (dh != 0.f || dlo != 0.f) {
        if (XLO) axpy2_df2(xh, xl, dh, dlo, rh, rl);
        else axpy2_df(xh, dh, dlo, rh, rl);
      }
      if (valid) {
        float* sn = snap + (size_t)(32 * m + i + 1) * 2 * a.ldw;
        __stcg(reinterpret_cast<float2*>(sn) + g2, rh);
        __stcg(reinterpret_cast<float2*>(sn + a.ldw) + g2, rl);
      }
    };
    auto ldx2 = [&](int i, int pl) {
      float2 x = *slot_of(buf, i, pl);
      if (!in0) x.x = 0.f;
      if (!in1) x.y = 0.f;
      return x;
    };
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {
      float2 xh[4], xl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xh[u] = ldx2(i + u, 0);
        xl[u] = XLO ? ldx2(i + u, 1) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) step(i + u, xh[u], xl[u]);
    }
    for (; i < cnt; ++i) step(i, ldx2(i, 0), XLO ? ldx2(i, 1) : make_float2(0.f, 0.f));
    __syncwarp();
    if (part == 0 && tid == 0) ctl->gprof[5] += (unsigned long long)(clock64() - tw1);
  }
  cp_async_wait<0>();
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
  __shared__ int gflags[16];
  __shared__ int s_vnext;  // one-CTA problems: next batch of positions a verifying warp takes

  // G CTAs cooperate on one problem: the whole grid, or a group of the batch
  const int G = BATCH ? a.gsize : (int)gridDim.x;
  const int cta = (int)blockIdx.x % G, grp = (int)blockIdx.x / G;
  // the single path's flow of rounds (planned rounds, Gram or direct form,
  // snapshot 0 as the residual): the single path and groups of CTAs of the
  // batched solver; one-CTA problems keep the residual in registers
  const bool SP = !BATCH || G > 1;
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
    if (!grid_sync(bc, bg, err, (unsigned)G, a.wait_ns, !BATCH)) goto fail; \
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
          ctl->aud_bits = 0ull;
          ctl->aud_tc_bits = 0ull;
          ctl->prob = atomicAdd(a.queue, 1);
        }
        if (!grid_sync(bc, bg, err, (unsigned)G, a.wait_ns)) break;
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
          if (tid == 0) {
            ctl->failed = 0;
            ctl->t_cur = 0;
            ctl->resume = 0;
            ctl->pdone = 0;
          }
          __syncthreads();
        } else if (vload(ctl->failed) != 0 || (a.pass_mode && vload(ctl->pdone) != 0)) {
          continue;  // its records were stamped when it failed, or its path is finished
        }
      } else if (G == 1) {
        batch_setup<XLO>(a, ctl, wsb, b, dbuf, 0, a.p, true, true, true);
      } else {
        // every CTA: the columns of its slice; CTA 0: y, rho and ||y||^2, then lambda_max
        batch_setup<XLO>(a, ctl, wsb, b, dbuf, f0, f1, false, cta == 0, false);
        if (!grid_sync(bc, bg, err, (unsigned)G, a.wait_ns)) goto fail;
        if (cta == 0) batch_setup<XLO>(a, ctl, wsb, b, dbuf, 0, 0, false, false, true);
        if (!grid_sync(bc, bg, err, (unsigned)G, a.wait_ns)) goto fail;
      }
      if (prof_thread && (!a.lockstep || a.t0 == 0)) {
        for (int k = 0; k < 8; ++k) ctl->prof[k] = 0ull;
        for (int k = 0; k < 8; ++k) ctl->gprof[k] = 0ull;
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
    const uint8_t* prm = (BATCH && a.rmask != nullptr) ? a.rmask + (size_t)b * a.ldm : nullptr;
    if (vload(*err) != 0) goto fail;  // NaN/Inf input or lambda_max = 0

  // pass mode: the problem continues at its own lambda, inside it when the
  // last launch ended after a pass (resume); c~ of the product is valid until
  // the residual changes in this launch (a pass, or a restart at a new lambda)
  const bool PM = BATCH && a.lockstep && a.pass_mode;
  const int t_begin = (BATCH && a.lockstep) ? (PM ? vload(ctl->t_cur) : a.t0) : 0;
  const int t_end = (BATCH && a.lockstep) ? (PM ? a.T : a.t1) : a.T;
  bool resume = PM && vload(ctl->resume) != 0;
  bool cvalid = BATCH && a.cfirst != nullptr;
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
    // per-lambda table lambda / ||x_j||^2; full mask; optional restart (a
    // resumed lambda has them from its first launch)
    if (!resume)
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
    if (!resume)
      for (int w = wd0 + tid; w < wd1; w += kThreads) {
        const int lo = w * 32, hi = min(a.p, lo + 32);
        WS(uint32_t, mask)[w] = (hi - lo == 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
      }
    if (cta == 0 && t > 0 && !a.warm_start && !resume)
      for (int i = tid; i < a.ldw; i += kThreads) {
        WS(float, rho_h)[i] = __ldcg(WS(float, rho0_h) + i);
        WS(float, rho_l)[i] = __ldcg(WS(float, rho0_l) + i);
      }
    // the product of a pass-mode launch was taken on the residual before this restart
    if (PM && t > 0 && !a.warm_start && !resume) cvalid = false;
    long long epochs = 0, checks = 0, xcols = 0;
    int scope_n = a.p;  // X^T rho scope of the next check
    // pass mode: the next pass of the period when the lambda resumes, else the check first
    int e_first = 0;
    bool skip_check = false;
    if (resume) {
      epochs = vload(ctl->ep_s);
      checks = vload(ctl->ck_s);
      xcols = vload(ctl->xc_s);
      scope_n = vload(ctl->scope_s);
      e_first = vload(ctl->e_cur);
      skip_check = e_first < a.f && epochs < a.max_epochs;
      if (!skip_check) e_first = 0;
    }
    if (PM && cta == 0 && tid == 0) ctl->t_cur = t;
    GSYNC();

    for (;;) {
      if (!skip_check) {
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
          double aud = 0.0, aud_tc = 0.0;
          // the first check of a lambda of a lockstep batch takes c~ from the
          // batched tensor-core product, with its own error factor
          const bool from_gemm = cvalid && (PM || checks == 0);
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
              if (a.audit) {
                // the exact correlation (double-float residual, exact sum) against c~ and its bound
                const df2 ce = warp_dot_exact<NG, XLO>(cx, j, WS(float, rho_h), WS(float, rho_l),
                                                       __fmul_ru(__ldcg(WS(float, nrmf) + j), rnormf));
                double cv = df_to_double(ce);
                if constexpr (EN) cv = __dsub_rn(cv, ridge_exact(j));
                const double ratio = fabs(__dsub_rn((double)c, cv)) / (double)E;
                if (from_gemm) aud_tc = fmax(aud_tc, ratio);
                else aud = fmax(aud, ratio);
              }
            }
            if (lane == 0) WS(float, ctil)[j] = c;
          }
          if (lane == 0) atomicMax(&ctl->mlo_bits, __float_as_uint(fmaxf(mlo, 0.f)));
          if (a.audit && lane == 0) {
            atomicMax(&ctl->aud_bits, (unsigned long long)__double_as_longlong(aud));
            atomicMax(&ctl->aud_tc_bits, (unsigned long long)__double_as_longlong(aud_tc));
          }
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
            st.bound_ratio = __longlong_as_double((long long)vload(ctl->aud_bits));
            st.bound_ratio_tc = __longlong_as_double((long long)vload(ctl->aud_tc_bits));
            ctl->aud_bits = 0ull;
            ctl->aud_tc_bits = 0ull;
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
              WS(float, dref)[kpos] = 0.f;
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
          ctl->anorm = rnormf;
        }
        // the anchor of the distance bound: the residual of this check
        if (!SP)
          for (int i = tid; i < a.ldw; i += kThreads) WS(float, anchor)[i] = __ldcg(WS(float, rho_h) + i);
        scope_n = a.xtr_scope == 0 ? a.p : totk;
        GSYNC();
        PROF(0);
      } else {
        // (P0) pass mode, a resumed lambda: the certificates of the zero
        // coefficients are issued anew from the product's c~ of the residual
        // this pass starts from (the rule of the check's certificates, with
        // the product's error factor), and the movement bound restarts at 0.
        // Without a product the certificates of the last pass stand.
        PROF(7);
        if (cvalid) {
          double rr = 0.0;
          for (int i = tid; i < a.n; i += kThreads) {
            const double r = __dadd_rn((double)__ldcg(WS(float, rho_h) + i), (double)__ldcg(WS(float, rho_l) + i));
            rr = __fma_rn(r, r, rr);
          }
          rr = block_sum_d(rr, dbuf);
          const float rnormf = __fmul_ru(__fsqrt_ru(__double2float_ru(rr)), 1.0001f);
          const float lam_lo = __fmul_rd(__double2float_rd(lam), 1.0f - 1e-6f);
          const int q = vload(ctl->q);
          // four positions per thread and step, their loads issued together
          for (int k0 = tid; k0 < q; k0 += 4 * kThreads) {
            int jj[4];
            float2 bb[4];
            float nn[4], cc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = k0 + u * kThreads;
              jj[u] = k < q ? __ldcg(WS(int, A) + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              bb[u] = ld_beta(cx, jj[u]);
              nn[u] = __ldcg(WS(float, nrmf) + jj[u]);
              cc[u] = __ldcg(a.cfirst + (size_t)jj[u] + (size_t)b * a.ldc);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = k0 + u * kThreads;
              if (k >= q) break;
              float sk = kSkChain;
              if (!nonzero2(bb[u])) {
                const float E = __fmul_ru(__fmul_ru(a.cfactor, nn[u]), rnormf) + 1e-37f;
                const float slack = __fsub_rd(lam_lo, __fadd_ru(fabsf(cc[u]), E));
                sk = (slack > 0.f && nn[u] > 0.f) ? __fdiv_rd(slack, nn[u]) : kSkNone;
              }
              WS(float, sk)[k] = sk;
              WS(float, mref)[k] = 0.f;
              WS(float, dref)[k] = 0.f;
            }
          }
          for (int i = tid; i < a.ldw; i += kThreads) WS(float, anchor)[i] = __ldcg(WS(float, rho_h) + i);
          __syncthreads();
          if (tid == 0) {
            ctl->mcur = 0.f;
            ctl->anorm = rnormf;
          }
        }
        GSYNC();
        PROF(0);
      }
      // ======================= PASSES =======================
      {
        const int q = vload(ctl->q);
        int s = vload(ctl->s);
        // a check's compaction writes sup0; a resumed pass continues with the list in use
        const bool par = skip_check && vload(ctl->sup_par) != 0;
        int* sup = par ? WS(int, sup1) : WS(int, sup0);
        int* sup_next = par ? WS(int, sup0) : WS(int, sup1);
        // Planning of a round (single path, CTA 0): the chain = [forced
        // entry] + the support positions of the window [pos, pos + win) (at
        // most s_cap of them).  The round ends at the window's end, or at the
        // first support position left out.  The round runs in Gram form when
        // the cache is in use and holds (or can take) every chain entry; the
        // bound on ||rho|| of its snapshots comes from snapshot 0.
        auto plan_round = [&](const int* supl, int s_cnt) {
          const int si = vload(ctl->sup_idx), forced = vload(ctl->forced), pos0 = vload(ctl->pos);
          const int plim = (int)min((long long)q, (long long)pos0 + vload(ctl->win));
          int below = 0;
          for (int i = si + tid; i < s_cnt; i += kThreads) below += (__ldcg(supl + i) < plim) ? 1 : 0;
          const int in_win = block_sum_i(below, ibuf);
          const int take = min(in_win, a.s_cap - (forced >= 0 ? 1 : 0));
          const int ncp = take + (forced >= 0 ? 1 : 0);
          const int next = (si + take < s_cnt) ? __ldcg(supl + si + take) : q;
          const int rend = take < in_win ? next : min(plim, next);
          for (int c = tid; c < ncp; c += kThreads)
            WS(int, chain)[c] = (forced >= 0) ? (c == 0 ? forced : __ldcg(supl + si + c - 1)) : __ldcg(supl + si + c);
          // Every coefficient of the support has a slot while the cache is in
          // use; an entering feature (the forced entry) gets a new one.  When a
          // round runs in direct form with an entering feature that has no
          // slot (the cache is full, or the chain is longer than a Gram round
          // holds), that feature joins the support without one, so the cache
          // is switched off for the rest of the lambda.
          int mode = 0, nsl = -1;
          bool full = false;
          if (a.gram_cap > 0 && vload(ctl->gram_on) != 0) {
            bool need = false;
            const int ns = vload(ctl->nslots);
            if (forced >= 0) {
              const int jf = __ldcg(WS(int, A) + forced);
              const int sl = __ldcg(WS(int, slot) + jf);
              need = !(sl >= 0 && sl < ns && __ldcg(WS(int, feat) + sl) == jf);
            }
            if (ncp > 0 && ncp <= kGramMaxNc && (!need || ns < a.gram_cap)) {
              mode = 1;
              if (need) nsl = ns;
            } else if (need) {
              full = true;
            }
          }
          __syncthreads();
          load_rho_regs<NGC, CW>(cx, WS(float, snap), WS(float, snap) + a.ldw, rh, rl);
          const float rbp = rho_bound_from_regs<NGC, EN>(cx, rh, lam, ncp, fbuf, rdg);
          if (tid == 0) {
            ctl->nc = ncp;
            ctl->round_end = rend;
            ctl->fstar = kNoPos;
            WS(float, msnap)[0] = ctl->mcur;
            ctl->rho_bound = rbp;
            ctl->pub_g = 0;
            ctl->rmode = mode;
            ctl->newslot = nsl;
            // an entering feature without a slot: the cache no longer covers
            // the support, so the rest of this lambda runs in direct form
            if (full) ctl->gram_on = 0;
          }
          __threadfence();
          __syncthreads();
        };
        // copy of snapshot e into snapshot 0 (the residual a round starts from) by CTA 0
        auto snap_to_front = [&](int e) {
          if (e <= 0) return;
          const float4* src = reinterpret_cast<const float4*>(WS(float, snap) + (size_t)e * 2 * a.ldw);
          float4* dst = reinterpret_cast<float4*>(WS(float, snap));
          for (int i = tid; i < 2 * a.ld4; i += kThreads) __stcg(dst + i, __ldcg(src + i));
        };
        // The Gram cache of the lambda (single path): after the first check
        // the slots 0..s-1 hold the support in ascending feature order, and
        // G[i][k] = x_i^T x_k for every pair of them (all CTAs)
        if (SP && a.gram_cap > 0 && checks == 1) {
          if (s > a.gram_cap) {
            if (cta == 0 && tid == 0) {
              ctl->gram_on = 0;
              ctl->nslots = 0;
            }
          } else {
            if (cta == 0) {
              for (int i = tid; i < s; i += kThreads) {
                const int j = __ldcg(WS(int, A) + __ldcg(sup + i));
                WS(int, feat)[i] = j;
                WS(int, slot)[j] = i;
              }
              if (tid == 0) {
                ctl->gram_on = 1;
                ctl->nslots = s;
              }
            }
            const long long pairs = (long long)s * (s - 1) / 2;
            float2* Gm = WS(float2, gram);
            for (long long t = cta * nwarps + warp; t < pairs; t += (long long)G * nwarps) {
              int i, k;
              tri_index(t, i, k);
              const int ji = __ldcg(WS(int, A) + __ldcg(sup + i)), jk = __ldcg(WS(int, A) + __ldcg(sup + k));
              const df2 v = warp_dot_cols<NG, XLO>(a.Xh + (long long)ji * a.ldx, XLO ? a.Xl + (long long)ji * a.ldx : nullptr,
                                                   a.Xh + (long long)jk * a.ldx, XLO ? a.Xl + (long long)jk * a.ldx : nullptr,
                                                   a.ld4, a.n, prm);
              if (lane == 0) {
                Gm[(size_t)i * a.gram_cap + k] = make_float2(v.h, v.l);
                Gm[(size_t)k * a.gram_cap + i] = make_float2(v.h, v.l);
              }
            }
          }
          GSYNC();
        }
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
        if (SP) {
          // the first round of the first pass (the residual of the removal is in snapshot 0)
          if (cta == 0) {
            __syncthreads();
            if (tid == 0) {
              ctl->pos = 0;
              ctl->sup_idx = 0;
              ctl->forced = -1;
              ctl->n_entered = 0;
            }
            __syncthreads();
            plan_round(sup, s);
          }
          GSYNC();
        }
        for (int e = e_first; e < a.f && epochs < a.max_epochs; ++e) {
          // ---- one pass over the safe-active list, in rounds
          if (!SP && cta == 0) {
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
            if (!SP) {
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
            } else {
              const int rmode = vload(ctl->rmode), ncr = vload(ctl->nc);
              if (rmode == 1) {
                // R1a (all CTAs): x_c^T rho_0 for every chain entry, and the
                // Gram row of an entering feature against the cache's slots
                const int newslot = vload(ctl->newslot);
                const int items = ncr + (newslot > 0 ? newslot : 0);
                const float* s0h = WS(float, snap);
                for (int it = cta * nwarps + warp; it < items; it += G * nwarps) {
                  if (it < ncr) {
                    const int j = __ldcg(WS(int, A) + __ldcg(WS(int, chain) + it));
                    const df2 v = warp_dot_col_rho<NG, XLO>(a.Xh + (long long)j * a.ldx,
                                                            XLO ? a.Xl + (long long)j * a.ldx : nullptr, s0h,
                                                            s0h + a.ldw, a.ld4, a.n);
                    if (lane == 0) WS(float2, g0)[it] = make_float2(v.h, v.l);
                  } else {
                    const int k = it - ncr;
                    const int jf = __ldcg(WS(int, A) + __ldcg(WS(int, chain))), jk = __ldcg(WS(int, feat) + k);
                    const df2 v = warp_dot_cols<NG, XLO>(a.Xh + (long long)jf * a.ldx,
                                                         XLO ? a.Xl + (long long)jf * a.ldx : nullptr,
                                                         a.Xh + (long long)jk * a.ldx,
                                                         XLO ? a.Xl + (long long)jk * a.ldx : nullptr, a.ld4, a.n,
                                                         prm);
                    if (lane == 0) {
                      WS(float2, gram)[(size_t)newslot * a.gram_cap + k] = make_float2(v.h, v.l);
                      WS(float2, gram)[(size_t)k * a.gram_cap + newslot] = make_float2(v.h, v.l);
                    }
                  }
                }
                GSYNC();
                // R1b: the chain in Gram form (CTA 0) and the snapshots (CTAs 1..nsc)
                if (cta == 0)
                  gram_round<NG, XLO, EN>(a, wsb, ctl, dsm, gflags, ncr, newslot, df_from_double(rdg), err);
                else if (cta <= a.nsc)
                  snapshot_follow<XLO>(a, wsb, ctl, dsm, ncr, cta - 1, err, prm);
              } else if (cta == 0 && ncr > 0) {
                if (prof_thread) ctl->gprof[7] += 1ull;
                // R1 in direct form (CTA 0), from snapshot 0
                load_rho_regs<NGC, CW>(cx, WS(float, snap), WS(float, snap) + a.ldw, rh, rl);
                run_chain<NGC, CW, XLO, EN>(cx, cs, ring, jl, ncr, vload(ctl->rho_bound), rh, rl, rbits,
                                            df_from_double(rdg));
              }
              if (cta == 0) {
                __threadfence();
                if (prof_thread) ctl->prof[5] += (unsigned long long)ncr;
              }
            }
            PROF(1);
            GSYNC();
            // R2 (all CTAs): the zero coefficients of [pos, round_end) must stay zero
            {
              const int pos = vload(ctl->pos), rend = vload(ctl->round_end), nc = vload(ctl->nc);
              const float rb = vload(ctl->rho_bound);
              const int span = rend - pos;
              // one-CTA problems: D_c >= ||rho_c - rho_a||, a bound on the
              // distance of snapshot c of the round from the anchor rho_a, and
              // the largest of them.  FP32 over the high planes: the sum of
              // squares is enlarged by its accumulation error ((terms per lane
              // + 8) 2^-23), its root by 1e-4 (the differences' rounding), and
              // 2^-22 (||rho_c|| + ||rho_a||) covers the dropped low planes (each
              // below 2^-24 of its high plane)
              float dmax = 3.0e38f;
              const long long td0 = clock64();
              if (!SP) {
                const float4* anc = reinterpret_cast<const float4*>(WS(float, anchor));
                const float abs_t = __fmul_ru(2.384185791015625e-07f, __fadd_ru(rb, vload(ctl->anorm)));
                const float fac = __fadd_ru(1.0f, __fmul_ru((float)(4 * ((a.ld4 + 31) / 32) + 8), 1.1920929e-07f));
                for (int c = warp; c <= nc; c += nwarps) {
                  const float4* sh = reinterpret_cast<const float4*>(WS(float, snap) + (size_t)c * 2 * a.ldw);
                  float S = 0.f;
                  for (int g = lane; g < a.ld4; g += 32) {
                    const float4 x = __ldcg(sh + g), y = __ldcg(anc + g);
                    const float d0 = __fsub_rn(x.x, y.x), d1 = __fsub_rn(x.y, y.y);
                    const float d2 = __fsub_rn(x.z, y.z), d3 = __fsub_rn(x.w, y.w);
                    S = __fmaf_rn(d0, d0, S);
                    S = __fmaf_rn(d1, d1, S);
                    S = __fmaf_rn(d2, d2, S);
                    S = __fmaf_rn(d3, d3, S);
                  }
                  S = warp_sum_f(S);
                  if (lane == 0)
                    WS(float, dsnap)[c] = __fadd_ru(__fmul_ru(__fsqrt_ru(__fmul_ru(S, fac)), 1.0001f), abs_t);
                }
                if (tid == 0) s_vnext = 0;
                __syncthreads();
                float m = 0.f;
                for (int c = lane; c <= nc; c += 32) m = fmaxf(m, __ldcg(WS(float, dsnap) + c));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                dmax = m;
                if (tid == 0) {
                  ctl->gprof[0] += 1ull;
                  ctl->gprof[4] += (unsigned long long)(clock64() - td0);
                }
              }
              unsigned long long n_scan = 0, n_read = 0, n_exact = 0;
              if (span > 0) {
                // a zero coefficient whose certificate survives the movement of
                // the residual since it was issued stays zero without a read:
                // |x_j^T rho| <= lambda - slack + ||x_j|| ||rho - rho_ref|| < lambda,
                // with ||rho - rho_ref|| <= M_now - M_ref (the movement counter)
                // and, for one-CTA problems, <= D_max + D_ref (both distances
                // from the anchor, the triangle inequality)
                const float mend = __ldcg(WS(float, msnap) + nc);
                const float* skp = WS(float, sk);
                float* mrp = WS(float, mref);
                // positions: the group's CTAs split the window into one
                // contiguous chunk per warp; the warps of a one-CTA problem take
                // batches of 32 positions in ascending order from a counter in
                // shared memory (the reads the certificates leave are unevenly
                // spread over the window), the next batch while this one is
                // processed.  A batch a warp holds when it stops lies past the
                // first entering position, where no verdict is needed.
                int i0s = pos, i1s = rend;
                if (SP) {
                  const int gw = cta * nwarps + warp, nwg = G * nwarps;
                  const int chunk = (span + nwg - 1) / nwg;
                  i0s = pos + gw * chunk;
                  i1s = min(rend, i0s + chunk);
                }
                // chain entries before the current batch of positions
                int sb = lower_bound_i(WS(int, chain), nc, i0s);
                float4 r4[NG];
                int loaded = -1;
                const float lamf = __double2float_rn(lam);
                const float lam_lo = __fmul_rd(__double2float_rd(lam), 1.0f - 1e-6f);
                // the verdict for position i (feature j, norm nf) from its FP32
                // correlation c with snapshot sg: stays zero (certificate
                // renewed) or enters
                auto decide = [&](int i, int j, float nf, float c, int sg, float ms, float ds) -> bool {
                  const float* sh = WS(float, snap) + (size_t)sg * 2 * a.ldw;
                  const float E = __fmul_ru(__fmul_ru(bf, nf), rb) + 1e-37f;
                  bool enters;
                  if (__fadd_ru(fabsf(c), E) < lamf * (1.0f - 1e-6f)) enters = false;
                  else if (__fsub_rd(fabsf(c), E) > lamf * (1.0f + 1e-6f)) enters = true;
                  else {
                    ++n_exact;
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
                    mrp[i] = ms;
                    if (!SP) WS(float, dref)[i] = ds;
                  }
                  return enters;
                };
                bool stop_warp = false;
                int bidx = SP ? 0 : __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(&s_vnext, 1) : 0, 0);
                for (;;) {
                  const int base = i0s + 32 * bidx;
                  if (base >= i1s || stop_warp) break;
                  if (SP) ++bidx;
                  else bidx = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(&s_vnext, 1) : 0, 0);
                  const int i1 = i1s;
                  const int il = base + lane;
                  n_scan += 32;
                  // the certificate test, with the feature of the position read
                  // alongside (used when the test fails)
                  bool need = false;
                  int jn = 0;
                  if (il < i1) {
                    const float sk = __ldcg(skp + il);
                    const float mr = __ldcg(mrp + il);
                    const float dr = SP ? 0.f : __ldcg(WS(float, dref) + il);
                    jn = __ldcg(WS(int, A) + il);
                    float mv = __fsub_ru(mend, mr);
                    if (!SP) mv = fminf(mv, __fadd_ru(dmax, dr));
                    need = !(mv < sk);
                  }
                  unsigned needm = __ballot_sync(0xffffffffu, need);
                  if (needm == 0u) continue;
                  // fstar moves under other warps' atomicMin: one lane reads it
                  // so that the whole warp takes the same branches.  A value
                  // that is stale by the end of the batch only costs work: a
                  // verdict past the first entering position is undone with
                  // the round, and the certificates it renews stay valid
                  const int fs = __shfl_sync(0xffffffffu, vload(ctl->fstar), 0);
                  if (base + __ffs(needm) - 1 > fs) break;
                  const float nfn = need ? __ldcg(WS(float, nrmf) + jn) : 0.f;
                  // the snapshot of each lane's position: the chain entries
                  // before it, sb (entries before base) plus those of the
                  // batch below it (a search over the ascending entries held
                  // one per lane; at most 31 of them lie in the batch)
                  for (;;) {
                    const int ce = (sb + lane < nc) ? __ldcg(WS(int, chain) + sb + lane) : 0x7fffffff;
                    const unsigned lt = __ballot_sync(0xffffffffu, ce < base);
                    sb += __popc(lt);
                    if (lt != 0xffffffffu) break;
                  }
                  const int ce = (sb + lane < nc) ? __ldcg(WS(int, chain) + sb + lane) : 0x7fffffff;
                  int cnt = 0;
#pragma unroll
                  for (int st = 16; st > 0; st >>= 1)
                    if (__shfl_sync(0xffffffffu, ce, cnt + st - 1) < il) cnt += st;
                  const int segl = sb + cnt;
                  // movement and distance of each needed lane's snapshot, for a renewal
                  const float msn = need ? __ldcg(WS(float, msnap) + segl) : 0.f;
                  const float dsn = (need && !SP) ? __ldcg(WS(float, dsnap) + segl) : 0.f;
                  while (needm) {
                    const int l = __ffs(needm) - 1;
                    needm &= needm - 1;
                    const int i = base + l;
                    if (i > fs) {
                      stop_warp = true;
                      break;
                    }
                    const int j = __shfl_sync(0xffffffffu, jn, l), sg = __shfl_sync(0xffffffffu, segl, l);
                    const float nf = __shfl_sync(0xffffffffu, nfn, l);
                    const float ms = __shfl_sync(0xffffffffu, msn, l), ds = __shfl_sync(0xffffffffu, dsn, l);
                    if (loaded != sg) {
                      const float* sh = WS(float, snap) + (size_t)sg * 2 * a.ldw;
#pragma unroll
                      for (int k = 0; k < NG; ++k) {
                        const int g = lane + 32 * k;
                        r4[k] = (g < a.ld4) ? ldcg4(sh, g) : make_float4(0.f, 0.f, 0.f, 0.f);
                      }
                      loaded = sg;
                    }
                    // the next needed position shares the snapshot when no chain
                    // entry lies between them: verify both with one pass of loads
                    // (up to 8 granules per lane; longer columns keep one)
                    constexpr bool kPair = NG <= 8;
                    const int l2 = needm ? __ffs(needm) - 1 : 0;
                    const int sg2 = __shfl_sync(0xffffffffu, segl, l2);
                    if (kPair && needm && sg2 == sg && base + l2 <= fs) {
                      const int j2 = __shfl_sync(0xffffffffu, jn, l2);
                      const float nf2 = __shfl_sync(0xffffffffu, nfn, l2);
                      const float ms2 = __shfl_sync(0xffffffffu, msn, l2), ds2 = __shfl_sync(0xffffffffu, dsn, l2);
                      float c, c2;
                      n_read += 2;
                      warp_dot_f32_2<NG>(a.Xh + (long long)j * a.ldx, a.Xh + (long long)j2 * a.ldx, r4, a.ld4, a.n,
                                         c, c2);
                      if (decide(i, j, nf, c, sg, ms, ds)) {
                        stop_warp = true;
                        break;
                      }
                      needm &= needm - 1;
                      if (decide(base + l2, j2, nf2, c2, sg, ms2, ds2)) {
                        stop_warp = true;
                        break;
                      }
                    } else {
                      ++n_read;
                      const float c = warp_dot_f32<NG>(a.Xh + (long long)j * a.ldx, r4, a.ld4, a.n);
                      if (decide(i, j, nf, c, sg, ms, ds)) {
                        stop_warp = true;
                        break;
                      }
                    }
                  }
                }
              }
              // one-CTA problems: positions scanned, columns read, exact refinements
              if (!SP && lane == 0) {
                atomicAdd(&ctl->gprof[1], n_scan);
                atomicAdd(&ctl->gprof[2], n_read);
                atomicAdd(&ctl->gprof[3], n_exact);
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
                if (SP) snap_to_front(nc);
              } else {
                // chain entries before the entering position stand; later ones are undone
                if (prof_thread) ctl->prof[6] += 1ull;
                const int seg = lower_bound_i(WS(int, chain), nc, fst);
                for (int c = seg + tid; c < nc; c += kThreads) WS(float2, bdf)[__ldcg(WS(int, A) + __ldcg(WS(int, chain) + c))] = WS(float2, oldb)[c];
                if (!SP) {
                  const float* sh = WS(float, snap) + (size_t)seg * 2 * a.ldw;
                  load_rho_regs<NGC, CW>(cx, sh, sh + a.ldw, rh, rl);
                } else {
                  snap_to_front(seg);
                }
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
              // the next round of the pass (single path)
              if (SP && vload(ctl->done) == 0) plan_round(sup, s);
            }
            GSYNC();
            PROF(3);
            if (vload(ctl->done)) break;
          }
          // end of pass (CTA 0): write rho; next support list = survivors of the
          // old list merged with the entered positions (both ascending)
          if (cta == 0) {
            if (!SP) store_rho_regs<NGC, CW>(cx, WS(float, rho_h), WS(float, rho_l), rh, rl);
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
            // single path: the first round of the next pass, if one follows
            if (SP && e + 1 < a.f && epochs + 1 < a.max_epochs) {
              if (tid == 0) {
                ctl->pos = 0;
                ctl->sup_idx = 0;
                ctl->forced = -1;
                ctl->n_entered = 0;
              }
              __syncthreads();
              plan_round(sup_next, nsurv + ne);
            }
          }
          ++epochs;
          xcols += q;
          GSYNC();
          PROF(4);
          s = vload(ctl->s);
          int* tmp = sup;
          sup = sup_next;
          sup_next = tmp;
          if (PM) {
            // pass mode: the launch ends for this problem after one pass; the
            // next launch resumes here with c~ of the new residual
            if (tid == 0) {
              ctl->resume = 1;
              ctl->e_cur = e + 1;
              ctl->ep_s = epochs;
              ctl->ck_s = checks;
              ctl->xc_s = xcols;
              ctl->scope_s = scope_n;
              ctl->sup_par = sup == WS(int, sup1) ? 1 : 0;
            }
            __syncthreads();
            goto pass_exit;
          }
        }
      }
      GSYNC();
      skip_check = false;
      e_first = 0;
    }
    // the lambda is finished: a later lambda of this launch starts afresh
    resume = false;
    if (PM && cta == 0 && tid == 0) ctl->resume = 0;
    if (PM && a.park && t + 1 < t_end) {
      if (tid == 0) {
        ctl->pdone = 1;
        a.park_t[b] = t + 1;
        atomicSub(a.active, 1);
      }
      __syncthreads();
      goto pass_exit;
    }
  }  // lambda loop
  if (PM && tid == 0) {
    ctl->pdone = 1;
    atomicSub(a.active, 1);
  }
    }
  pass_exit:
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
      if (G > 1) grid_sync(bc, bg, err, (unsigned)G, a.wait_ns);
      if (cta == 0) {
        lasso_path_stats* so = a.stats + (size_t)b * a.T;
        const int tf0 = a.lockstep ? (a.pass_mode ? vload(ctl->t_cur) : a.t0) : 0;
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
          if (a.lockstep && a.pass_mode) atomicSub(a.active, 1);
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

template <int NGC, int CW, bool XLO, bool BATCH, int MINB = 1, bool EN = false>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&path_kernel<NGC, CW, XLO, BATCH, MINB, EN>);
}

// Host-side pointers of the kernel's instantiations.  Each group is compiled
// in a translation unit of its own (path_k_*.cu) so that the build runs them
// in parallel.  ngc: float4 granules per chain lane (1, 2 or 4); cw: chain
// warps (1 or 4).
const void* path_kernel_single_f32(int ngc, int cw);
const void* path_kernel_single_f64(int ngc, int cw);
const void* path_kernel_enet(int ngc, int cw);
const void* path_kernel_enet_f64(int ngc, int cw);
const void* path_kernel_batch(int ngc, int per_sm);
const void* path_kernel_batch_enet(int ngc, int per_sm);

}  // namespace lassogs
