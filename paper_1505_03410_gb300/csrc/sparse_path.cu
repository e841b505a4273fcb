// Lasso paths on a sparse design in compressed-column (CSC) storage: the
// sparse variant of the solver of Sec. 4.1 (the paper's implementation has a
// dense Fortran-ordered and a sparse CSC version).  Algorithm 1 as in the
// dense path: a GAP SAFE check every f passes (Eq. (7), (10); the dome of
// Eq. (11) and the radius of Thm. 2 as options), warm starts along the grid
// of Sec. 3.3, stop when the gap is <= eps; the Elastic-Net of the appendix
// as the Lasso on [X; sqrt(mu) I] with the extra rows implicit.
//
// On sparse data the work is gathers and scatters over the nonzeros, not
// flops, so the arithmetic is FP64 throughout:
//   check   (all CTAs)  c_j = x_j^T rho, one warp per column gathering rho over
//                       the column's nonzeros; objectives, gap, radius and the
//                       test in every CTA from the same reductions (fixed
//                       order, so every CTA takes the same decisions)
//   removal (CTA 0)     screened nonzero coefficients set to zero and their
//                       share added back to rho, in ascending j (Remark 3)
//   passes  (CTA 0)     cyclic coordinate descent over the safe-active list,
//                       rho in shared memory; warp 0 gathers x_j^T rho,
//                       updates beta_j and scatters the update into rho
// The order of every residual update is the oracle's, so the iterates are
// Algorithm 1's up to the rounding of the n-long sums.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "internal.h"

namespace lassogs {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpMaxGrid = 1024;
constexpr int64_t kSpMaxRows = 16384;  // rows: the residual lives in shared memory during the passes

__device__ __forceinline__ unsigned long long vload_ull(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ long long vload_ll(const long long* p) {
  return *reinterpret_cast<const volatile long long*>(p);
}

// a device error (invalid input, a wait that timed out) into every record
__global__ void sparse_stats_error_kernel(const int* err, lasso_path_stats* stats, int T) {
  const int e = *err;
  if (e == 0) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    stats[t].status = e;
    stats[t].converged = 0;
  }
}

struct SpCtrl {
  unsigned bar_count, bar_gen;
  int err;
  int bad_input;
  unsigned long long m_bits;  // max |c_j| over the scope (FP64 bits)
  double lambda_max, yy, eps;
  int q;      // safe-active count after the last check
  int nzl;    // coefficients the last check removed
  long long passes;
};

struct SpArgs {
  const int64_t* colptr;
  const int32_t* rowidx;
  const double* val;
  int n, p, T, words, f;
  int dual_point, xtr_scope, warm_start, screen_rule, refined_radius;
  double enet_alpha, tol;
  long long max_epochs;
  unsigned long long wait_ns;
  const double* y;
  const double* ratios;
  const double* beta0;
  double* beta_out;
  uint32_t* mask_out;
  lasso_path_stats* stats;
  // workspace
  SpCtrl* ctl;
  double *beta, *rho, *rho0, *nrm2, *cy, *c, *part, *zl;
  uint32_t *mask, *zbits;
  int* A;
};

// x_j^T v over the nonzeros of column j (whole warp, all lanes get the sum)
__device__ __forceinline__ double col_dot(const SpArgs& a, int j, const double* v) {
  const int lane = threadIdx.x & 31;
  const long long k0 = a.colptr[j], k1 = a.colptr[j + 1];
  double s = 0.0;
  for (long long k = k0 + lane; k < k1; k += 32) s = __fma_rn(a.val[k], v[a.rowidx[k]], s);
  return warp_sum_d(s);
}

__device__ __forceinline__ double dome_value(double xc, double rad, double al, double xnr, double xn) {
  // support function of the dome (center c, radius rad, normal, ratio al) at x,
  // from c^T x, nrm^T x and ||x||: the ball's extreme point when it lies in the
  // dome, else the maximum over the circle where the hyperplane cuts the sphere
  if (xnr < __dmul_rn(-al, xn)) return __dadd_rn(xc, __dmul_rn(rad, xn));
  double w = __dsub_rn(__dmul_rn(xn, xn), __dmul_rn(xnr, xnr));
  if (w < 0.0) w = 0.0;
  return __dadd_rn(__dsub_rn(xc, __dmul_rn(__dmul_rn(rad, al), xnr)),
                   __dmul_rn(rad, __dsqrt_rn(__dmul_rn(w, __dsub_rn(1.0, __dmul_rn(al, al))))));
}

__global__ void __launch_bounds__(kSpThreads, 1) sparse_path_kernel(SpArgs a) {
  extern __shared__ __align__(16) double srho[];  // n doubles: rho during the passes (CTA 0)
  __shared__ double dbuf[32];
  __shared__ int ibuf[32];
  const int G = (int)gridDim.x, cta = (int)blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kSpThreads / 32;
  SpCtrl* ctl = a.ctl;
  unsigned* bc = &ctl->bar_count;
  unsigned* bg = &ctl->bar_gen;
  int* err = &ctl->err;
  const double u64 = 1.1102230246251565e-16;  // 2^-53
  const double ea = a.enet_alpha;
  const bool enet = ea < 1.0;
  // feature slice of this CTA (32-aligned, so that mask words belong to one CTA)
  const int fs = ((a.p + G - 1) / G + 31) / 32 * 32;
  const int f0 = min(a.p, cta * fs), f1 = min(a.p, f0 + fs);
  const int wd0 = f0 >> 5, wd1 = f1 > f0 ? (f1 + 31) >> 5 : wd0;
#define SGSYNC()                                                     \
  do {                                                               \
    if (!grid_sync(bc, bg, err, (unsigned)G, a.wait_ns, true)) return; \
  } while (0)

  // ---- set-up: ||x_j||^2, x_j^T y (lambda_max, Sec. 1.2), input checks; rho = y - X beta0
  for (int j = f0 + warp; j < f1; j += nwarps) {
    const long long k0 = a.colptr[j], k1 = a.colptr[j + 1];
    bool ok = k1 >= k0;
    double s2 = 0.0, sy = 0.0;
    for (long long k = k0 + lane; ok && k < k1; k += 32) {
      const int r = a.rowidx[k];
      const double v = a.val[k];
      if (r < 0 || r >= a.n || !isfinite(v)) {
        ok = false;
        break;
      }
      s2 = __fma_rn(v, v, s2);
      sy = __fma_rn(v, a.y[r], sy);
    }
    ok = __all_sync(0xffffffffu, ok);
    s2 = warp_sum_d(s2);
    sy = warp_sum_d(sy);
    if (lane == 0) {
      if (!ok) atomicExch(&ctl->bad_input, 1);
      a.nrm2[j] = s2;
      a.cy[j] = sy;
      if (ok && isfinite(sy)) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(fabs(sy)));
      a.beta[j] = a.beta0 ? a.beta0[j] : 0.0;
    }
  }
  if (cta == 0) {
    for (int i = tid; i < a.n; i += kSpThreads) srho[i] = a.y[i];
    __syncthreads();
    if (a.beta0 != nullptr && warp == 0) {
      // rho = y - X beta0, the nonzero terms subtracted in ascending j (the oracle's order)
      for (int j = 0; j < a.p; ++j) {
        const double b = a.beta0[j];
        if (b == 0.0) continue;
        const long long k0 = a.colptr[j], k1 = a.colptr[j + 1];
        for (long long k = k0 + lane; k < k1; k += 32) {
          const int r = a.rowidx[k];
          if (r >= 0 && r < a.n) srho[r] = __dsub_rn(srho[r], __dmul_rn(b, a.val[k]));
        }
        __syncwarp();
      }
    }
    __syncthreads();
    double yy = 0.0;
    for (int i = tid; i < a.n; i += kSpThreads) {
      a.rho[i] = srho[i];
      a.rho0[i] = srho[i];
      yy = __fma_rn(a.y[i], a.y[i], yy);
    }
    yy = block_sum_d(yy, dbuf);
    if (tid == 0) {
      ctl->yy = yy;
      ctl->eps = a.tol * yy;
    }
  }
  SGSYNC();
  if (cta == 0 && tid == 0) {
    ctl->lambda_max = __ddiv_rn(__longlong_as_double((long long)vload_ull(&ctl->m_bits)), ea);
    bool bad = !(ctl->lambda_max > 0.0) || ctl->bad_input;
    for (int t = 0; t < a.T; ++t) bad = bad || !(a.ratios[t] > 0.0 && a.ratios[t] <= 1.0);
    if (bad) ctl->err = 1;  // LASSO_ERR_INVALID_ARG
    ctl->m_bits = 0ull;
  }
  SGSYNC();
  if (ld_volatile(err) != 0) return;
  const double yy = ctl->yy, eps = ctl->eps, lmax = ctl->lambda_max;

  for (int t = 0; t < a.T; ++t) {
    const double lam_path = __dmul_rn(lmax, a.ratios[t]);
    const double lam = __dmul_rn(ea, lam_path);                          // L1 weight
    const double mu = enet ? __dmul_rn(__dsub_rn(1.0, ea), lam_path) : 0.0;  // ridge weight
    for (int w = wd0 + tid; w < wd1; w += kSpThreads) {
      const int lo = w * 32, hi = min(a.p, lo + 32);
      a.mask[w] = (hi - lo == 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
    }
    if (t > 0 && !a.warm_start) {
      for (int j = f0 + tid; j < f1; j += kSpThreads) a.beta[j] = a.beta0 ? a.beta0[j] : 0.0;
      if (cta == 0)
        for (int i = tid; i < a.n; i += kSpThreads) a.rho[i] = a.rho0[i];
    }
    long long epochs = 0, checks = 0, xcols = 0;
    int scope_n = a.p;
    SGSYNC();
    for (;;) {
      // ================= CHECK: c = X^T rho over the scope, the maxima and norms
      double mloc = 0.0;
      for (int j = f0 + warp; j < f1; j += nwarps) {
        const bool in = a.xtr_scope == 0 || ((a.mask[j >> 5] >> (j & 31)) & 1u);
        double cj = 0.0;
        if (in) {
          cj = col_dot(a, j, a.rho);
          if (enet) cj = __dsub_rn(cj, __dmul_rn(mu, a.beta[j]));  // x~_j^T rho~
          mloc = fmax(mloc, fabs(cj));
        }
        if (lane == 0) a.c[j] = cj;
      }
      if (lane == 0) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(mloc));
      double l1p = 0.0, l2p = 0.0;
      for (int j = f0 + tid; j < f1; j += kSpThreads) {
        const double b = a.beta[j];
        l1p = __dadd_rn(l1p, fabs(b));
        l2p = __fma_rn(b, b, l2p);
      }
      l1p = block_sum_d(l1p, dbuf);
      l2p = block_sum_d(l2p, dbuf);
      if (tid == 0) {
        a.part[2 * cta] = l1p;
        a.part[2 * cta + 1] = l2p;
      }
      SGSYNC();
      // every CTA: the same scalars from the same sums in the same order
      double l1 = 0.0, l2 = 0.0;
      for (int c = tid; c < G; c += kSpThreads) {
        l1 = __dadd_rn(l1, a.part[2 * c]);
        l2 = __dadd_rn(l2, a.part[2 * c + 1]);
      }
      l1 = block_sum_d(l1, dbuf);
      l2 = block_sum_d(l2, dbuf);
      double rr = 0.0, yr = 0.0;
      for (int i = tid; i < a.n; i += kSpThreads) {
        const double r = a.rho[i];
        rr = __fma_rn(r, r, rr);
        yr = __fma_rn(a.y[i], r, yr);
      }
      rr = block_sum_d(rr, dbuf);
      yr = block_sum_d(yr, dbuf);
      if (enet) rr = __dadd_rn(rr, __dmul_rn(mu, l2));  // ||rho~||^2 = ||rho||^2 + mu ||beta||^2
      const double m = __longlong_as_double((long long)vload_ull(&ctl->m_bits));
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
      for (int i = tid; i < a.n; i += kSpThreads) {
        const double dd = __dsub_rn(__dmul_rn(lam, __dmul_rn(alpha, a.rho[i])), a.y[i]);
        d2 = __fma_rn(dd, dd, d2);
      }
      d2 = block_sum_d(d2, dbuf);
      if (enet) {
        const double la = __dmul_rn(lam, alpha);
        d2 = __dadd_rn(d2, __dmul_rn(__dmul_rn(la, la), __dmul_rn(mu, l2)));
      }
      const double P = __dadd_rn(__dmul_rn(0.5, rr), __dmul_rn(lam, l1));
      const double D = __dsub_rn(__dmul_rn(0.5, yy), __dmul_rn(0.5, d2));
      const double Gap = __dsub_rn(P, D);
      const double tau = 2.0 * (double)(a.n + a.p + (enet ? a.p : 0) + 8) * u64 * (rr + lam * l1 + yy + d2);
      const double Gs = (Gap > 0.0 ? Gap : 0.0) + tau;
      double rad = __ddiv_rn(__dsqrt_rn(__dmul_rn(2.0, Gs)), lam);
      if (a.refined_radius == 1) {
        const double Rt = __ddiv_rn(__dsqrt_rn(__dadd_rn(d2, tau)), lam);
        if (Rt < rad) rad = Rt;
      }
      const double aa = fabs(alpha);
      const bool dome = a.screen_rule == 1 && d2 > 0.0;
      double drad = 0.0, dal = 0.0, dR = 1.0;
      if (dome) {
        const double big = __dadd_rn(d2, tau);
        double small = __dsub_rn(__dsub_rn(yy, __dmul_rn(2.0, P)), tau);
        if (small < 0.0) small = 0.0;
        double qq = __ddiv_rn(small, big);
        if (qq > 1.0) qq = 1.0;
        dal = __dsub_rn(__dmul_rn(2.0, qq), 1.0);
        drad = __ddiv_rn(__dmul_rn(0.5, __dsqrt_rn(big)), lam);
        dR = __ddiv_rn(__dsqrt_rn(d2), lam);
      }
      ++checks;
      xcols += scope_n;
      const bool stop = Gap <= eps;
      const bool cap = epochs >= a.max_epochs;
      // the test (Eq. (7); with the dome, Eq. (11) as well) on the slice
      int kept = 0, nnz = 0;
      for (int w0 = f0 + 32 * warp; w0 < f1; w0 += 32 * nwarps) {
        const int j = w0 + lane;
        const bool valid = j < f1;
        const uint32_t word = a.mask[w0 >> 5];
        const bool was = valid && ((word >> lane) & 1u);
        bool keep = was;
        if (was) {
          double xn = __dsqrt_rn(a.nrm2[j]);
          if (enet) xn = __dsqrt_rn(__dadd_rn(a.nrm2[j], mu));
          const double cj = a.c[j];
          const double muj = __dadd_rn(__dmul_rn(fabs(cj), aa), __dmul_rn(rad, xn));
          keep = !(muj < 1.0);
          if (keep && dome) {
            const double xt = __dmul_rn(alpha, cj);
            const double xy = __ddiv_rn(a.cy[j], lam);
            const double xc = __dmul_rn(0.5, __dadd_rn(xy, xt));
            const double xnr = __ddiv_rn(__dsub_rn(xy, xt), dR);
            const double md = fmax(dome_value(xc, drad, dal, xnr, xn), dome_value(-xc, drad, dal, -xnr, xn));
            if (md < 1.0) keep = false;
          }
        }
        const double bj = valid ? a.beta[j] : 0.0;
        const bool zeroed = was && !keep && bj != 0.0 && !stop && !cap;
        if (zeroed) {
          a.zl[j] = bj;
          a.beta[j] = 0.0;
        }
        const uint32_t zw = __ballot_sync(0xffffffffu, zeroed);
        const uint32_t nwd = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) {
          a.mask[w0 >> 5] = nwd;
          a.zbits[w0 >> 5] = zw;
        }
        kept += __popc(nwd);
        nnz += __popc(__ballot_sync(0xffffffffu, valid && (zeroed ? false : bj != 0.0)));
      }
      if (lane != 0) kept = nnz = 0;
      kept = block_sum_i(kept, ibuf);
      nnz = block_sum_i(nnz, ibuf);
      if (tid == 0) {
        reinterpret_cast<int*>(a.part + 2 * kSpMaxGrid)[2 * cta] = kept;
        reinterpret_cast<int*>(a.part + 2 * kSpMaxGrid)[2 * cta + 1] = nnz;
      }
      if (cta == 0 && tid == 0) ctl->m_bits = 0ull;
      SGSYNC();
      if (stop || cap) {
        for (int j = f0 + tid; j < f1; j += kSpThreads) a.beta_out[(long long)t * a.p + j] = a.beta[j];
        if (a.mask_out)
          for (int w = wd0 + tid; w < wd1; w += kSpThreads) a.mask_out[(long long)t * a.words + w] = a.mask[w];
        if (cta == 0) {
          int totk = 0, totn = 0;
          for (int c = tid; c < G; c += kSpThreads) {
            totk += reinterpret_cast<const int*>(a.part + 2 * kSpMaxGrid)[2 * c];
            totn += reinterpret_cast<const int*>(a.part + 2 * kSpMaxGrid)[2 * c + 1];
          }
          totk = block_sum_i(totk, ibuf);
          totn = block_sum_i(totn, ibuf);
          if (tid == 0) {
            lasso_path_stats st{};
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
            st.status = stop ? 0 : 5;
            a.stats[t] = st;
          }
        }
        SGSYNC();
        break;
      }
      // ================= removal, compaction and passes (CTA 0)
      if (cta == 0) {
        for (int i = tid; i < a.n; i += kSpThreads) srho[i] = a.rho[i];
        __syncthreads();
        if (warp == 0) {
          // rho += b x_j for the removed coefficients, ascending j
          for (int w = 0; w < a.words; ++w) {
            uint32_t zw = a.zbits[w];
            while (zw) {
              const int j = w * 32 + __ffs(zw) - 1;
              zw &= zw - 1;
              const double b = a.zl[j];
              const long long k0 = a.colptr[j], k1 = a.colptr[j + 1];
              for (long long k = k0 + lane; k < k1; k += 32) {
                const int r = a.rowidx[k];
                srho[r] = __dadd_rn(srho[r], __dmul_rn(b, a.val[k]));
              }
              __syncwarp();
            }
          }
        }
        // ascending safe-active list
        int q = 0;
        for (int base = 0; base < a.words; base += kSpThreads) {
          const int w = base + tid;
          const uint32_t word = w < a.words ? a.mask[w] : 0u;
          const int cnt = __popc(word);
          // exclusive prefix of the counts over the block
          int incl = cnt;
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          if (lane == 31) ibuf[warp] = incl;
          __syncthreads();
          int before = q;
          for (int ww = 0; ww < warp; ++ww) before += ibuf[ww];
          before += incl - cnt;
          uint32_t wd = word;
          int k = 0;
          while (wd) {
            const int b = __ffs(wd) - 1;
            wd &= wd - 1;
            a.A[before + k++] = w * 32 + b;
          }
          int tot = 0;
          for (int ww = 0; ww < nwarps; ++ww) tot += ibuf[ww];
          __syncthreads();
          q += tot;
        }
        __syncthreads();
        // f passes of cyclic coordinate descent over A (Algorithm 1)
        long long done = 0;
        if (warp == 0) {
          for (int e = 0; e < a.f && epochs + done < a.max_epochs; ++e) {
            for (int ii = 0; ii < q; ++ii) {
              const int j = a.A[ii];
              const double nr = enet ? __dadd_rn(a.nrm2[j], mu) : a.nrm2[j];
              if (!(nr > 0.0)) continue;
              double g = col_dot(a, j, srho);
              const double bj = a.beta[j];
              if (enet) g = __dsub_rn(g, __dmul_rn(mu, bj));
              const double b = __dadd_rn(bj, __ddiv_rn(g, nr));
              const double thr = __ddiv_rn(lam, nr);
              const double nb = b > thr ? __dsub_rn(b, thr) : (b < -thr ? __dadd_rn(b, thr) : 0.0);
              if (nb != bj) {
                const double d = __dsub_rn(nb, bj);
                const long long k0 = a.colptr[j], k1 = a.colptr[j + 1];
                for (long long k = k0 + lane; k < k1; k += 32) {
                  const int r = a.rowidx[k];
                  srho[r] = __dsub_rn(srho[r], __dmul_rn(d, a.val[k]));
                }
                if (lane == 0) a.beta[j] = nb;
              }
              __syncwarp();
            }
            ++done;
          }
        }
        __syncthreads();
        for (int i = tid; i < a.n; i += kSpThreads) a.rho[i] = srho[i];
        if (tid == 0) {
          ctl->q = q;
          ctl->passes = done;
        }
        __threadfence();
      }
      SGSYNC();
      const long long done = vload_ll(&ctl->passes);
      const int q = ld_volatile(&ctl->q);
      epochs += done;
      xcols += (long long)q * done;
      scope_n = a.xtr_scope == 0 ? a.p : q;
    }
  }
#undef SGSYNC
}

}  // namespace
}  // namespace lassogs

using namespace lassogs;

extern "C" size_t lasso_path_csc_workspace_size(int64_t n, int64_t p, const lasso_opts* opts) {
  (void)opts;
  if (n < 1 || n > kSpMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4) return 0;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t words = (size_t)(p + 31) / 32;
  return al(sizeof(SpCtrl)) + 5 * al(sizeof(double) * p) + 2 * al(sizeof(double) * n) +
         al(sizeof(double) * 2 * kSpMaxGrid + sizeof(int) * 2 * kSpMaxGrid) + 2 * al(sizeof(uint32_t) * words) +
         al(sizeof(int) * p) + al(sizeof(double) * p);
}

extern "C" lasso_status lasso_path_csc(const int64_t* colptr, const int32_t* rowidx, const double* values, int64_t n,
                                       int64_t p, const double* y, const double* ratios, int32_t T,
                                       const double* beta0, const lasso_opts* opts, double* beta_out,
                                       uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                                       void* stream_) {
  clear_error();
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_default_opts(&o);
  lasso_status st = check_options(o);
  if (st != LASSO_OK) return st;
  if (!colptr || !y || !ratios || !beta_out || !stats || (!rowidx && p > 0) || (!values && p > 0))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_csc: colptr, rowidx, values, y, lambda_ratios, beta_out and "
                                            "stats must be non-NULL");
  if (n < 1 || n > kSpMaxRows)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_csc: need 1 <= n <= %lld", (long long)kSpMaxRows);
  if (p < 1 || p > (int64_t)INT32_MAX / 4) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_csc: p out of range");
  if (T < 1) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_csc: T must be >= 1");
  auto aligned = [](const void* q, uintptr_t k) { return (reinterpret_cast<uintptr_t>(q) % k) == 0; };
  if (!aligned(colptr, 8) || !aligned(rowidx, 4) || !aligned(values, 8) || !aligned(y, 8) || !aligned(ratios, 8) ||
      !aligned(beta_out, 8) || !aligned(stats, 8) || (beta0 && !aligned(beta0, 8)) || (mask_out && !aligned(mask_out, 4)))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_csc: misaligned argument");
  const size_t need = lasso_path_csc_workspace_size(n, p, &o);
  if (!ws || !aligned(ws, 256)) return set_error(LASSO_ERR_WORKSPACE, "lasso_path_csc: workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need)
    return set_error(LASSO_ERR_WORKSPACE, "lasso_path_csc: workspace of %zu bytes < %zu required", ws_bytes, need);
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  char* base = static_cast<char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = base + off;
    off += al(bytes);
    return q;
  };
  SpArgs a{};
  a.colptr = colptr;
  a.rowidx = rowidx;
  a.val = values;
  a.n = (int)n;
  a.p = (int)p;
  a.T = T;
  a.words = (int)((p + 31) / 32);
  a.f = o.screen_period;
  a.dual_point = o.dual_point;
  a.xtr_scope = o.xtr_scope;
  a.warm_start = o.warm_start;
  a.screen_rule = o.screen_rule;
  a.refined_radius = o.refined_radius;
  a.enet_alpha = o.enet_alpha;
  a.tol = o.gap_tol_rel;
  a.max_epochs = o.max_epochs;
  a.wait_ns = wait_limit_ns();
  a.y = y;
  a.ratios = ratios;
  a.beta0 = beta0;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  a.ctl = reinterpret_cast<SpCtrl*>(take(sizeof(SpCtrl)));
  a.beta = reinterpret_cast<double*>(take(sizeof(double) * p));
  a.nrm2 = reinterpret_cast<double*>(take(sizeof(double) * p));
  a.cy = reinterpret_cast<double*>(take(sizeof(double) * p));
  a.c = reinterpret_cast<double*>(take(sizeof(double) * p));
  a.zl = reinterpret_cast<double*>(take(sizeof(double) * p));
  a.rho = reinterpret_cast<double*>(take(sizeof(double) * n));
  a.rho0 = reinterpret_cast<double*>(take(sizeof(double) * n));
  a.part = reinterpret_cast<double*>(take(sizeof(double) * 2 * kSpMaxGrid + sizeof(int) * 2 * kSpMaxGrid));
  a.mask = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * a.words));
  a.zbits = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * a.words));
  a.A = reinterpret_cast<int*>(take(sizeof(int) * p));
  int dev = 0, sms = 0, coop = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return set_error(LASSO_ERR_CUDA, "device does not support cooperative launch");
  const size_t dyn = sizeof(double) * (size_t)n;
  const void* kfn = reinterpret_cast<const void*>(&sparse_path_kernel);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int occ = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kSpThreads, dyn));
  if (occ < 1) return set_error(LASSO_ERR_CUDA, "the sparse path kernel cannot be resident");
  const int grid = std::min(sms, kSpMaxGrid);
  CUDA_TRY(cudaMemsetAsync(a.ctl, 0, sizeof(SpCtrl), stream));
  void* params[] = {&a};
  CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kSpThreads), params, dyn, stream));
  sparse_stats_error_kernel<<<1, 128, 0, stream>>>(&a.ctl->err, stats, T);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}
