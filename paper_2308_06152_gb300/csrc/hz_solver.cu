// Host orchestration of the method and the C ABI of include/hz.h.
//
// The host only sequences kernel launches on the caller's stream and reads
// a few convergence flags; every arithmetic step runs in the kernels of
// hz_stencil.cu, hz_krylov.cu and hz_gradient.cu.  All device storage is
// carved out of the caller's workspace; the library never allocates device
// memory.
//
// Method (arXiv 2308.06152):
//   outer   flexible GMRES on A x = b, right-preconditioned (Sec. 6.3)
//   precond P_A-DEF1 v = M^-1 (v - A Q v) + Q v (Sec. 3.2.2, eq. ADEF1),
//           Q v = Z E^-1 R v with R = Z^T / 4 (Sec. 5.2, eqs. matvec-*)
//   E^-1    GMRES on E v2 = v1, right-preconditioned by a V-cycle on the
//           coarse CSLP (Sec. 5.2, Sec. 6)
//   M^-1    one V-cycle: damped Jacobi (w = 0.8) pre/post sweep, full
//           weighting, bilinear interpolation, re-discretised coarse CSLP,
//           direct coarsest solve (Sec. 3.1, 4, 5.1)
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "hz.h"
#include "hz_common.cuh"

using namespace hz;

namespace {

constexpr int kMaxLevels = 24;
constexpr int kMaxCoarsest = 1024;
constexpr int kMaxRhs = 1024;
constexpr int kMaxIters = 3000;   // Krylov basis size (Givens column in smem)
constexpr unsigned long long kPipelineWaitNs = 2000000000ull;   // bounded waits

struct LevelHost {
  int nx = 0, ny = 0;
  long long n = 0;
  double h = 0;
  double* k2d = nullptr;
  float* k2f = nullptr;
  double2* dinv_d = nullptr;
  float2* dinv_f = nullptr;
  void* f = nullptr;   // level right-hand side (levels >= 1)
  void* x = nullptr;   // level solution (levels >= 1)
  void* xa = nullptr;  // pre-smoothed iterate (all levels)
  LevelDev dev() const {
    LevelDev d;
    d.nx = nx;
    d.ny = ny;
    d.h = h;
    d.ih2d = 1.0 / (h * h);
    d.tihd = 2.0 / h;
    d.ih2f = (float)d.ih2d;
    d.tihf = (float)d.tihd;
    d.k2d = k2d;
    d.k2f = k2f;
    d.dinv_d = dinv_d;
    d.dinv_f = dinv_f;
    return d;
  }
};

struct Arena {
  char* base = nullptr;
  size_t off = 0;
  bool dry = true;
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = dry ? nullptr : base + off;
    off += bytes;
    return p;
  }
};

bool valid_desc(const hz_desc* d, std::string* why) {
  if (!d) { *why = "null descriptor"; return false; }
  if (d->nx < 3 || d->ny < 3) { *why = "grid needs at least 3 x 3 nodes"; return false; }
  if (!(d->h > 0)) { *why = "h must be positive"; return false; }
  if (d->bc != HZ_BC_DIRICHLET && d->bc != HZ_BC_SOMMERFELD) { *why = "bad bc"; return false; }
  if (d->zkind < HZ_Z_NONE || d->zkind > HZ_Z_HO) { *why = "bad zkind"; return false; }
  if (d->ekind < HZ_E_GALERKIN || d->ekind > HZ_E_RED_9PT) { *why = "bad ekind"; return false; }
  if (d->prec < HZ_PREC_FP64 || d->prec > HZ_PREC_MIXED_BF16) { *why = "bad prec"; return false; }
  if (d->nrhs_max < 1 || d->nrhs_max > kMaxRhs) { *why = "nrhs_max must be in 1..1024"; return false; }
  if (d->outer_maxit < 1 || d->coarse_maxit < 1 || d->outer_maxit > kMaxIters ||
      d->coarse_maxit > kMaxIters) {
    *why = "iteration caps must be in 1..3000";
    return false;
  }
  if (d->min_coarse_intervals < 1) { *why = "min_coarse_intervals must be >= 1"; return false; }
  if (!(d->jacobi_omega > 0)) { *why = "jacobi_omega must be positive"; return false; }
  if (d->outer_solver != HZ_OUTER_FGMRES && d->outer_solver != HZ_OUTER_GCR) {
    *why = "bad outer_solver";
    return false;
  }
  if (d->preconditioner != HZ_PRECOND_ADEF1 && d->preconditioner != HZ_PRECOND_TLKM) {
    *why = "bad preconditioner";
    return false;
  }
  if (d->preconditioner == HZ_PRECOND_TLKM && d->zkind == HZ_Z_NONE) {
    *why = "TLKM needs deflation vectors";
    return false;
  }
  if (d->deflation_levels < 0 || d->deflation_levels >= kMaxLevels ||
      (d->deflation_levels >= 2 &&
       (d->zkind == HZ_Z_NONE || d->preconditioner != HZ_PRECOND_ADEF1))) {
    *why = "deflation_levels must be 0/1, or 2 .. 23 with deflation vectors and A-DEF1";
    return false;
  }
  if (d->restart < 0 || d->restart > d->outer_maxit ||
      (d->restart > 0 && d->outer_solver != HZ_OUTER_FGMRES)) {
    *why = "restart must be in 0 .. outer_maxit (FGMRES only)";
    return false;
  }
  if (d->deflation_scaling != HZ_DEFL_SCALE_CONSISTENT &&
      (d->deflation_scaling != HZ_DEFL_SCALE_PRINTED || d->deflation_levels >= 2)) {
    *why = "deflation_scaling must be CONSISTENT, or PRINTED with at most two levels";
    return false;
  }
  return true;
}

std::vector<std::pair<int, int>> level_shapes(int nx, int ny, int min_ci) {
  std::vector<std::pair<int, int>> s{{nx, ny}};
  while ((int)s.size() < kMaxLevels) {
    const int cx = s.back().first, cy = s.back().second;
    if ((cx - 1) % 2 || (cy - 1) % 2) break;
    const int ncx = (cx - 1) / 2 + 1, ncy = (cy - 1) / 2 + 1;
    if (ncx - 1 < min_ci || ncy - 1 < min_ci) break;
    s.push_back({ncx, ncy});
  }
  return s;
}

}  // namespace

struct hz_solver {
  hz_desc d{};
  cudaStream_t st = nullptr;
  int L = 0;
  LevelHost lv[kMaxLevels];
  bool mixed = false;
  bool lvbf16 = false;   // V-cycle level vectors stored as BF16 pairs
  size_t esz = 16;       // bytes of one complex value of the preconditioner
  size_t lsz = 16;       // bytes of one stored value of a V-cycle level vector
  int nL = 0;            // unknowns of the dense coarsest level
  void* minv = nullptr;  // coarsest inverse, preconditioner precision
  double2* aug = nullptr;
  int* gj_err = nullptr;
  // preconditioner scratch (preconditioner precision), fine level
  void *fz1 = nullptr, *t = nullptr, *yv = nullptr, *q = nullptr,
       *vin = nullptr;
  // coarse level (level 1)
  void *v1 = nullptr, *v2 = nullptr, *sb = nullptr, *eb = nullptr, *Qb = nullptr;
  void* qf = nullptr;      // current basis vector in compute precision (FP16 basis)
  void* Sglk = nullptr;    // stcl-op-Glk coefficient planes [P*P][n1] (Galerkin E)
  // multilevel deflation (deflation_levels = D >= 2): the Krylov solve of
  // the coarse system E_l v2 = v1 of every deflation level l = 1 .. D.
  // Level 1's basis, state and vectors are Qb, kin, qf, sb, eb above; its
  // flexible directions and A-DEF1 vectors are in dl[1].  Levels below 1
  // keep their bases in compute precision.
  struct DefLevel {
    KState ks{};
    void *Q = nullptr, *Zb = nullptr;
    void *v1 = nullptr, *v2 = nullptr, *qf = nullptr, *sb = nullptr, *eb = nullptr;
    void *zj = nullptr, *q = nullptr, *u = nullptr;
  };
  bool ml = false;
  int D = 1;
  DefLevel dl[kMaxLevels];
  bool basis16 = false;    // inner Krylov basis stored as FP16 pairs
  KState kin{}, kout{};
  int* in_total = nullptr;
  int* in_max = nullptr;
  int* out_total = nullptr;   // outer iterations of finished restart cycles
  int* out_max = nullptr;     // (scratch of the accumulation)
  // outer FGMRES (FP64)
  double2 *Vo = nullptr, *Zo = nullptr, *wo = nullptr;
  double2* ro = nullptr;   // GCR residual
  double2* xg = nullptr;   // GCR iterate (the solver's own, so graphs can hold it)
  int* izero = nullptr;    // a device 0 (column index of a one-vector dot)
  double* bnorm_o = nullptr;
  double* relres = nullptr;
  // host-buffer solve and gradient storage
  double2 *io0 = nullptr, *io1 = nullptr, *io2 = nullptr;
  double* Jd = nullptr;
  int check_every = 4;
  std::string err;
  size_t ws_bytes = 0;
  // opt-in per-kernel-class timing (hz_profile_begin / hz_profile_end)
  unsigned long long* prof_bytes = nullptr;
  int prof_kc = HZ_KC_NONE;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
  long long prof_dropped = 0;
  // CUDA graphs of one outer iteration, the inner loop as a WHILE node; one
  // per (nrhs, tol), captured on the library's own streams (stream capture
  // is not allowed on the legacy default stream) and launched on st
  struct OuterGraph {
    int nrhs;
    double tol;
    int step;            // -1: an FGMRES iteration; k: GCR step k
    cudaGraph_t g;
    cudaGraphExec_t ex;
    long long kernels;   // kernels of one launch outside WHILE bodies
  };
  std::vector<OuterGraph> graphs;
  // whole solves captured for hz_solve_async, one per (nrhs, tol, use_x0,
  // buffers); the outer loop is a WHILE node (level 0) holding the inner one
  struct SolveGraph {
    int nrhs, use_x0;
    double tol;
    const void *b, *x, *info;
    cudaGraph_t g;
    cudaGraphExec_t ex;
    long long kernels;
  };
  std::vector<SolveGraph> solve_graphs;
  // (the WHILE body of deflation level l is captured on cap_body for
  // l = 1, on cap_nest[l] below it, and nested in its parent's body)
  cudaStream_t cap_main = nullptr, cap_body = nullptr;
  cudaStream_t cap_nest[kMaxLevels] = {};
  bool capturing = false;
  long long body_count = 0;      // kernels of all WHILE bodies, one pass each
  long long body_count_l[kMaxLevels] = {};   // own kernels of level l's body
  int* loop_it = nullptr;        // device [kMaxLevels]: iterations per loop
  int* body_kernels = nullptr;   // device [kMaxLevels]: body_count_l
  int* fault = nullptr;          // device: a Krylov pipeline wait timed out
  int* grp = nullptr;            // device [4]: flags of a group solve's graph
  hz_tuning tune{};
  int body_kernels_host[kMaxLevels] = {};

  ~hz_solver() {
    for (OuterGraph& g : graphs) {
      cudaGraphExecDestroy(g.ex);
      cudaGraphDestroy(g.g);
    }
    for (SolveGraph& g : solve_graphs) {
      cudaGraphExecDestroy(g.ex);
      cudaGraphDestroy(g.g);
    }
    if (cap_main) cudaStreamDestroy(cap_main);
    if (cap_body) cudaStreamDestroy(cap_body);
    for (cudaStream_t c : cap_nest)
      if (c) cudaStreamDestroy(c);
  }
};

namespace {

void set_err(hz_solver* s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
}

hz_status cuda_check(hz_solver* s, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(s, "%s: %s", where, cudaGetErrorString(e));
    return HZ_CUDA_ERROR;
  }
  return HZ_OK;
}

// Row stride of the inner Krylov basis: padded to 4 elements so that every
// row starts 16-byte aligned for the group loads of the Gram-Schmidt kernels.
inline long long inner_row(long long n) { return (n + 3) & ~3LL; }

KState plan_kstate(Arena& a, int B, int m, long long n) {
  KState k{};
  k.m = m;
  k.nblk_max = krylov_nblk(n);
  k.jctr = (int*)a.take(sizeof(int));
  k.alldone = (int*)a.take(sizeof(int));
  k.done = (int*)a.take(sizeof(int) * B);
  k.iters = (int*)a.take(sizeof(int) * B);
  k.stat = (int*)a.take(sizeof(int) * B);
  k.bnorm = (double*)a.take(sizeof(double) * B);
  k.beta = (double*)a.take(sizeof(double) * B);
  k.hnorm = (double*)a.take(sizeof(double) * B);
  k.H = (double2*)a.take(sizeof(double2) * (size_t)B * (m + 1) * m);
  k.g = (double2*)a.take(sizeof(double2) * (size_t)B * (m + 1));
  k.cs = (double*)a.take(sizeof(double) * (size_t)B * m);
  k.sn = (double2*)a.take(sizeof(double2) * (size_t)B * m);
  k.y = (double2*)a.take(sizeof(double2) * (size_t)B * m);
  k.hcol = (double2*)a.take(sizeof(double2) * (size_t)B * (m + 1));
  k.part = (double2*)a.take(sizeof(double2) * (size_t)B * (m + 1) * k.nblk_max);
  k.npart = (double*)a.take(sizeof(double) * (size_t)B * k.nblk_max);
  k.wpart = (double*)a.take(sizeof(double) * (size_t)B * k.nblk_max);
  k.reorth = (int*)a.take(sizeof(int) * B);
  k.fault = nullptr;   // set by plan(): one flag per solver
  k.dotk = 0;
  k.updk = 0;
  k.wait_ns = kPipelineWaitNs;
  k.starve = 0;
  return k;
}

// Assigns every device buffer of the solver inside the arena.
void plan(hz_solver* s, Arena& a) {
  const hz_desc& d = s->d;
  const int B = d.nrhs_max;
  const size_t es = s->esz;
  for (int l = 0; l <= s->L; ++l) {
    LevelHost& v = s->lv[l];
    v.k2d = (double*)a.take(sizeof(double) * v.n);
    v.k2f = s->mixed ? (float*)a.take(sizeof(float) * v.n) : nullptr;
    v.dinv_d = s->mixed ? nullptr : (double2*)a.take(sizeof(double2) * v.n);
    v.dinv_f = s->mixed ? (float2*)a.take(sizeof(float2) * v.n) : nullptr;
    v.xa = a.take(s->lsz * B * v.n);
    if (l >= 1) {
      v.f = a.take(s->lsz * B * v.n);
      v.x = a.take(s->lsz * B * v.n);
    }
  }
  s->minv = a.take(es * (size_t)s->nL * s->nL);
  s->aug = (double2*)a.take(sizeof(double2) * (size_t)s->nL * 2 * s->nL);
  s->gj_err = (int*)a.take(sizeof(int));
  const long long n0 = s->lv[0].n;
  s->t = a.take(es * B * n0);
  s->yv = a.take(es * B * n0);
  s->fz1 = d.preconditioner == HZ_PRECOND_TLKM ? a.take(es * B * n0) : nullptr;
  s->vin = s->mixed ? a.take(es * B * n0) : nullptr;
  if (d.zkind != HZ_Z_NONE) {
    const long long n1 = s->lv[1].n;
    s->q = a.take(es * B * n0);

    s->v1 = a.take(es * B * n1);
    s->v2 = a.take(es * B * n1);
    s->sb = a.take(es * B * n1);
    s->eb = a.take(es * B * n1);
    const size_t bes = s->basis16 ? sizeof(__half2) : es;
    s->Qb = a.take(bes * (size_t)B * inner_row(n1) * (d.coarse_maxit + 1));
    s->qf = a.take(es * B * n1);
    s->kin = plan_kstate(a, B, d.coarse_maxit, n1);
    if (d.ekind == HZ_E_GALERKIN) {
      const int P = d.zkind == HZ_Z_HO ? 5 : 3;
      s->Sglk = a.take(es * (size_t)P * P * n1);
    }
    if (s->ml) {
      const int m = d.coarse_maxit;
      for (int l = 1; l <= s->D; ++l) {
        hz_solver::DefLevel& D = s->dl[l];
        const long long nl = s->lv[l].n;
        if (l >= 2) {
          D.Q = a.take(es * (size_t)B * inner_row(nl) * (m + 1));
          D.ks = plan_kstate(a, B, m, nl);
          D.v1 = a.take(es * B * nl);
          D.v2 = a.take(es * B * nl);
          D.qf = a.take(es * B * nl);
          D.sb = a.take(es * B * nl);
          D.eb = a.take(es * B * nl);
        }
        if (l < s->D) {
          D.Zb = a.take(es * (size_t)B * nl * m);
          D.zj = a.take(es * B * nl);
          D.q = a.take(es * B * nl);
          D.u = a.take(es * B * nl);
        }
      }
    }
  }
  s->in_total = (int*)a.take(sizeof(int) * B);
  s->in_max = (int*)a.take(sizeof(int) * B);
  s->out_total = (int*)a.take(sizeof(int) * B);
  s->out_max = (int*)a.take(sizeof(int) * B);
  s->Vo = (double2*)a.take(sizeof(double2) * (size_t)B * n0 * (d.outer_maxit + 1));
  s->Zo = (double2*)a.take(sizeof(double2) * (size_t)B * n0 * d.outer_maxit);
  s->wo = (double2*)a.take(sizeof(double2) * (size_t)B * n0);
  s->kout = plan_kstate(a, B, d.outer_maxit, n0);
  s->bnorm_o = (double*)a.take(sizeof(double) * B);
  s->relres = (double*)a.take(sizeof(double) * B);
  s->io0 = (double2*)a.take(sizeof(double2) * (size_t)B * n0);
  s->io1 = (double2*)a.take(sizeof(double2) * (size_t)B * n0);
  s->io2 = (double2*)a.take(sizeof(double2) * (size_t)B * n0);
  s->Jd = (double*)a.take(sizeof(double));
  s->prof_bytes = (unsigned long long*)a.take(sizeof(unsigned long long));
  s->izero = (int*)a.take(sizeof(int));
  s->ro = d.outer_solver == HZ_OUTER_GCR
              ? (double2*)a.take(sizeof(double2) * (size_t)B * n0)
              : nullptr;
  s->xg = d.outer_solver == HZ_OUTER_GCR
              ? (double2*)a.take(sizeof(double2) * (size_t)B * n0)
              : nullptr;
  s->loop_it = (int*)a.take(sizeof(int) * kMaxLevels);
  s->body_kernels = (int*)a.take(sizeof(int) * kMaxLevels);
  s->fault = (int*)a.take(sizeof(int));
  s->grp = (int*)a.take(sizeof(int) * 4);
  s->kin.fault = s->fault;
  s->kout.fault = s->fault;
  for (int l = 2; l <= s->D; ++l) {
    s->dl[l].ks.fault = s->fault;
    s->dl[l].ks.dotk = s->tune.mdot_kernel;
    s->dl[l].ks.updk = s->tune.maxpy_kernel;
  }
  s->kin.dotk = s->kout.dotk = s->tune.mdot_kernel;
  s->kin.updk = s->kout.updk = s->tune.maxpy_kernel;
}

hz_status init_shapes(hz_solver* s) {
  const hz_desc& d = s->d;
  const auto sh = level_shapes(d.nx, d.ny, d.min_coarse_intervals);
  s->L = (int)sh.size() - 1;
  double h = d.h;
  for (int l = 0; l <= s->L; ++l) {
    s->lv[l].nx = sh[l].first;
    s->lv[l].ny = sh[l].second;
    s->lv[l].n = (long long)sh[l].first * sh[l].second;
    s->lv[l].h = h;
    h *= 2.0;
  }
  s->nL = (int)s->lv[s->L].n;
  if (d.zkind != HZ_Z_NONE && s->L < 1) {
    set_err(s, "deflation needs a grid that coarsens at least once "
               "(nx-1, ny-1 even, coarse intervals >= %d)", d.min_coarse_intervals);
    return HZ_INVALID_GRID;
  }
  if (s->nL > kMaxCoarsest) {
    set_err(s, "coarsest level has %d nodes; the dense coarsest solve allows "
               "at most %d (choose nx-1, ny-1 with more factors of 2)",
            s->nL, kMaxCoarsest);
    return HZ_INVALID_GRID;
  }
  s->mixed = d.prec != HZ_PREC_FP64;
  s->lvbf16 = d.prec == HZ_PREC_MIXED_BF16;
  s->esz = s->mixed ? sizeof(float2) : sizeof(double2);
  s->lsz = s->lvbf16 ? sizeof(__nv_bfloat162) : s->esz;
  s->basis16 = s->mixed && d.inner_basis_fp16;
  s->D = d.deflation_levels < 1 ? 1 : d.deflation_levels;
  s->ml = s->D >= 2;
  if (s->ml && s->L < s->D) {
    set_err(s, "deflation to level %d needs a grid that coarsens %d times", s->D, s->D);
    return HZ_INVALID_GRID;
  }
  return HZ_OK;
}

// CSLP coefficient as printed in Sec. 5.1: ap = (4 - (beta1 - beta2 i) k^2 h^2)
// / h^2, i.e. M = -Lap - (beta1 - i beta2) k^2 (with beta2 = -0.5 the shift
// damps with the same sign as the Sommerfeld rows).
inline Shift cslp(const hz_solver* s) { return Shift{s->d.beta1, -s->d.beta2}; }

// Deflation restriction scale (hz_defl_scale): 4 turns R_Z = Z^T / 4 into
// the printed Z^T, for re-discretised E only (the Galerkin E's deflation
// does not depend on the scale); the printed 5x5 ReD-Glk rows are 4 times
// those on the Z^T / 4 scale.
inline double rz_scale(const hz_solver* s) {
  return (s->d.deflation_scaling == HZ_DEFL_SCALE_PRINTED && s->d.ekind != HZ_E_GALERKIN)
             ? 4.0
             : 1.0;
}
inline double glk_scale(const hz_solver* s) {
  return s->d.deflation_scaling == HZ_DEFL_SCALE_PRINTED ? 4.0 : 1.0;
}
inline Shift helm1() { return Shift{1.0, 0.0}; }

// FP64 view of level l (k2d present at every level)
inline LevelDev dev64(const hz_solver* s, int l) { return s->lv[l].dev(); }

// launch-bracketing events of the live per-kernel profiler (hz_profile_*)
inline void prof_mark(hz_solver* s, int kc) {
  if (s->prof_kc != kc) return;
  if (s->prof_used < s->prof_ev.size())
    cudaEventRecord(s->prof_ev[s->prof_used++], s->st);
  else
    ++s->prof_dropped;
}

// ------------------------------------------------------------ V-cycle
// The first level ls > l0 from which the rest of the hierarchy (levels ls ..
// L, three vectors per level and two for the coarsest, in FP32) fits in the
// shared memory of one block: k_vcycle_small takes those levels in one
// launch.  Staged complex-FP32 V-cycles only, and only with at least one
// level besides the coarsest; otherwise L + 1 (none).
template <class T>
int small_from(const hz_solver* s, int l0) {
  if (!std::is_same<T, float>::value || s->tune.vcycle_fused != 2) return s->L + 1;
  if (s->L - l0 < 2 || s->L - l0 > kMaxSmallLevels) return s->L + 1;
  long long elems = 2LL * s->nL;
  int ls = s->L;
  while (ls - 1 > l0 && ls - 1 >= s->L - (kMaxSmallLevels - 1)) {
    const long long n = s->lv[ls - 1].n;
    if ((elems + 3 * n) * (long long)sizeof(float2) > kSmallLevelBytes) break;
    elems += 3 * n;
    --ls;
  }
  return ls < s->L ? ls : s->L + 1;
}
SmallLevels small_levels(const hz_solver* s, int ls) {
  SmallLevels d;
  std::memset(&d, 0, sizeof(d));
  d.nlev = s->L - ls + 1;
  d.bc = s->d.bc;
  d.nL = (int)s->nL;
  d.omc = (float)(1.0 - s->d.jacobi_omega);
  int off = 0;
  for (int k = 0; k < d.nlev; ++k) {
    d.lv[k] = s->lv[ls + k].dev();
    d.off[k] = off;
    off += (k + 1 < d.nlev ? 3 : 2) * (int)s->lv[ls + k].n;
  }
  d.bytes = off * (int)sizeof(float2);
  return d;
}

// One V-cycle from level l0 for M_l0 x = f.  The hierarchy's own vectors are
// stored as SL (C<T>, or BF16 pairs for the BF16-storage smoother); the
// input f and the result xout are C<T>.
template <class T, class SL, class SI = C<T>>
void vcycle_sl(hz_solver* s, int l0, VRefE<SI> f, C<T>* xout, int nrhs,
               const int* done, long long frs = 0) {
  // SI: storage of the input f (C<T>, or FP16 pairs read straight from the
  // inner Krylov basis, staged kernels only); frs: distance between its
  // right-hand sides (0 = the level's node count; the basis rows are padded)
  constexpr bool native_in = std::is_same<SI, C<T>>::value;
  cudaStream_t st = s->st;
  const int bc = s->d.bc;
  const Shift sh = cslp(s);
  const C<T>* minv = (const C<T>*)s->minv;
  if constexpr (native_in) {
    if (l0 == s->L) {
      launch_dense_mv<T, C<T>, C<T>>(s->nL, minv, f, xout, nrhs, done, st);
      return;
    }
  }
  const bool fused = s->tune.vcycle_fused != 0;
  const bool staged = s->tune.vcycle_fused == 2;
  const int rpb = s->tune.vcycle_rhs_per_block, tile = s->tune.vcycle_tile;
  const double om = s->d.jacobi_omega;
  unsigned long long* vbytes = s->prof_kc == HZ_KC_VCYCLE ? s->prof_bytes : nullptr;
  // levels from ls down in one launch (k_vcycle_small), if any
  const int ls = small_from<T>(s, l0);
  const int lend = ls <= s->L ? ls : s->L;
  for (int l = l0; l < lend; ++l) {
    const LevelHost& A = s->lv[l];
    const LevelHost& Bc = s->lv[l + 1];
    if (staged) {
      if (l == l0) {
        prof_mark(s, HZ_KC_VCYCLE);
        launch_pre_restrict_mr<T, SI, SL, SL>(A.dev(), Bc.dev(), bc, om, f, (SL*)A.xa,
                                              (SL*)Bc.f, nrhs, rpb, done, st, vbytes, frs);
        prof_mark(s, HZ_KC_VCYCLE);
      } else
        launch_pre_restrict_mr<T, SL, SL, SL>(A.dev(), Bc.dev(), bc, om, vrefe<SL>(A.f),
                                              (SL*)A.xa, (SL*)Bc.f, nrhs, rpb, done, st);
      continue;
    }
    if constexpr (native_in) {
      if (fused) {
        if (l == l0)
          launch_pre_restrict<T, C<T>, SL, SL>(A.dev(), Bc.dev(), bc, sh, f, (SL*)A.xa,
                                               (SL*)Bc.f, nrhs, done, st);
        else
          launch_pre_restrict<T, SL, SL, SL>(A.dev(), Bc.dev(), bc, sh, vrefe<SL>(A.f),
                                             (SL*)A.xa, (SL*)Bc.f, nrhs, done, st);
        continue;
      }
      if (l == l0) {
        launch_jacobi0<T, C<T>, SL>(A.dev(), bc, f, (SL*)A.xa, nrhs, done, st);
        launch_resid_restrict<T, C<T>, SL, SL>(A.dev(), Bc.dev(), bc, sh, f,
                                               (const SL*)A.xa, (SL*)Bc.f, nrhs,
                                               done, st);
      } else {
        const VRefE<SL> fl = vrefe<SL>(A.f);
        launch_jacobi0<T, SL, SL>(A.dev(), bc, fl, (SL*)A.xa, nrhs, done, st);
        launch_resid_restrict<T, SL, SL, SL>(A.dev(), Bc.dev(), bc, sh, fl,
                                             (const SL*)A.xa, (SL*)Bc.f, nrhs, done,
                                             st);
      }
    }
  }
  if (ls <= s->L) {
    if constexpr (std::is_same<T, float>::value)
      launch_vcycle_small<SL>(small_levels(s, ls), (const SL*)s->lv[ls].f, (SL*)s->lv[ls].x,
                              (const float2*)minv, nrhs, done, st);
  } else {
    launch_dense_mv<T, SL, SL>(s->nL, minv, vrefe<SL>(s->lv[s->L].f),
                               (SL*)s->lv[s->L].x, nrhs, done, st);
  }
  for (int l = lend - 1; l >= l0; --l) {
    const LevelHost& A = s->lv[l];
    const LevelHost& Bc = s->lv[l + 1];
    if (staged) {
      if (l == l0) {
        prof_mark(s, HZ_KC_VCYCLE);
        launch_prolong_smooth_mr<T, SL, SL, SI, C<T>>(A.dev(), Bc.dev(), bc, om,
                                                      (const SL*)Bc.x, (const SL*)A.xa, f,
                                                      xout, nrhs, rpb, tile, done, st, vbytes,
                                                      frs);
        prof_mark(s, HZ_KC_VCYCLE);
      } else
        launch_prolong_smooth_mr<T, SL, SL, SL, SL>(A.dev(), Bc.dev(), bc, om,
                                                    (const SL*)Bc.x, (const SL*)A.xa,
                                                    vrefe<SL>(A.f), (SL*)A.x, nrhs, rpb, tile,
                                                    done, st);
      continue;
    }
    if constexpr (native_in) {
      if (fused) {
        if (l == l0)
          launch_prolong_smooth<T, SL, SL, C<T>, C<T>>(A.dev(), Bc.dev(), bc, sh,
                                                       (const SL*)Bc.x, (const SL*)A.xa, f,
                                                       xout, nrhs, done, st);
        else
          launch_prolong_smooth<T, SL, SL, SL, SL>(A.dev(), Bc.dev(), bc, sh,
                                                   (const SL*)Bc.x, (const SL*)A.xa,
                                                   vrefe<SL>(A.f), (SL*)A.x, nrhs, done, st);
        continue;
      }
      launch_prolong_add<T, SL, SL>(A.dev(), Bc.dev(), bc, (const SL*)Bc.x, (SL*)A.xa,
                                    nrhs, done, st);
      if (l == l0)
        launch_smooth<T, C<T>, SL, C<T>>(A.dev(), bc, sh, f, (const SL*)A.xa, xout,
                                         nrhs, done, st);
      else
        launch_smooth<T, SL, SL, SL>(A.dev(), bc, sh, vrefe<SL>(A.f), (const SL*)A.xa,
                                     (SL*)A.x, nrhs, done, st);
    }
  }
}

// The inner solve's V-cycle reads the current basis vector straight from the
// FP16 basis (no FP32 copy is written): the two-level A-DEF1 inner solve
// with an FP16 basis and the staged V-cycle kernels, on a hierarchy below
// level 1.  (The input is then exactly the stored basis vector.)
inline bool inner_in16(const hz_solver* s) {
  return s->basis16 && s->tune.vcycle_fused == 2 && s->d.preconditioner == HZ_PRECOND_ADEF1 &&
         !s->ml && s->L > 1;
}

// One V-cycle from level l0 whose input f is stored as FP16 pairs (the
// current vector of the FP16 inner Krylov basis, read in place); the staged
// kernels only (hz_tuning.vcycle_fused = 2), with a level below l0.
void vcycle_in16(hz_solver* s, int l0, VRefE<__half2> f, float2* xout, int nrhs,
                 const int* done) {
  const long long frs = inner_row(s->lv[l0].n);
  if (s->lvbf16)
    vcycle_sl<float, __nv_bfloat162, __half2>(s, l0, f, xout, nrhs, done, frs);
  else
    vcycle_sl<float, float2, __half2>(s, l0, f, xout, nrhs, done, frs);
}

template <class T>
void vcycle(hz_solver* s, int l0, VRef<T> f, C<T>* xout, int nrhs, const int* done) {
  if constexpr (std::is_same<T, float>::value) {
    if (s->lvbf16) {
      vcycle_sl<T, __nv_bfloat162>(s, l0, f, xout, nrhs, done);
      return;
    }
  }
  vcycle_sl<T, C<T>>(s, l0, f, xout, nrhs, done);
}

// ------------------------------------------------------------ coarse E
template <class T>
void apply_E(hz_solver* s, const C<T>* x, C<T>* y, int nrhs, const int* done) {
  cudaStream_t st = s->st;
  const int bc = s->d.bc;
  const LevelHost& F = s->lv[0];
  const LevelHost& Cc = s->lv[1];
  switch (s->d.ekind) {
    case HZ_E_GALERKIN:
      if (s->tune.galerkin_apply == 1)
        launch_stencil_e<T>(Cc.dev(), s->d.zkind == HZ_Z_HO ? 2 : 1, s->tune.e_column_pairs,
                            (const C<T>*)s->Sglk, x, y, nrhs, s->tune.e_rhs_per_block,
                            done, st);
      else
        launch_galerkin_fused<T>(F.dev(), Cc.dev(), bc, s->d.zkind, x, y, nrhs, done,
                                 st);
      break;
    case HZ_E_RED_O2:
      launch_helm<T>(Cc.dev(), bc, helm1(), vref<T>(x), vref<T>(nullptr), y, nrhs,
                     done, st);
      break;
    case HZ_E_RED_GLK1:
      launch_glk<T>(Cc.dev(), bc, 1, x, y, nrhs, done, st, glk_scale(s));
      break;
    case HZ_E_RED_O4:
      launch_red_o4<T>(Cc.dev(), bc, x, y, nrhs, done, st);
      break;
    case HZ_E_RED_CMPO4:
      launch_red_cmpo4<T>(Cc.dev(), bc, x, y, nrhs, done, st);
      break;
    case HZ_E_RED_O6:
      launch_red_o6<T>(Cc.dev(), bc, x, y, nrhs, done, st);
      break;
    case HZ_E_RED_9PT:
      launch_red_9pt<T>(Cc.dev(), bc, x, y, nrhs, done, st);
      break;
    default:
      launch_glk<T>(Cc.dev(), bc, 2, x, y, nrhs, done, st, glk_scale(s));
      break;
  }
}

// stcl-op-Glk set-up: the coefficients of E = R_Z A_h Z by FP64 probing of
// the on-the-fly product (the outer basis, unused until a solve, holds the
// probes and their images).
void extract_galerkin_stencil(hz_solver* s) {
  cudaStream_t st = s->st;
  const int P = s->d.zkind == HZ_Z_HO ? 5 : 3, K = P * P;
  const long long n1 = s->lv[1].n;
  const size_t scratch = sizeof(double2) * (size_t)s->d.nrhs_max * s->lv[0].n *
                         (s->d.outer_maxit + 1);
  long long pb = (long long)(scratch / (2 * sizeof(double2) * (size_t)n1));
  if (pb > K) pb = K;
  double2* pin = s->Vo;
  double2* pout = s->Vo + pb * n1;
  const LevelDev F = dev64(s, 0), Cc = dev64(s, 1);
  for (int c0 = 0; c0 < K; c0 += (int)pb) {
    const int nb = (int)(K - c0 < pb ? K - c0 : pb);
    launch_probe_fill(Cc, P, c0, nb, pin, st);
    launch_galerkin_fused<double>(F, Cc, s->d.bc, s->d.zkind, pin, pout, nb, nullptr, st);
    if (s->mixed)
      launch_probe_extract<float>(Cc, P, c0, nb, pout, (float2*)s->Sglk, st);
    else
      launch_probe_extract<double>(Cc, P, c0, nb, pout, (double2*)s->Sglk, st);
  }
}

hz_status read_flag(hz_solver* s, const int* dptr, int* out) {
  if (cudaMemcpyAsync(out, dptr, sizeof(int), cudaMemcpyDeviceToHost, s->st) !=
      cudaSuccess)
    return cuda_check(s, "flag copy");
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return cuda_check(s, "flag sync");
  return HZ_OK;
}

// The outer loop's stopping flag, raised also when a Krylov kernel's bounded
// wait ran out (the fault stays set for the report, which returns HZ_TIMEOUT).
hz_status read_outer_flag(hz_solver* s, int* out) {
  int v[2] = {0, 0};
  if (cudaMemcpyAsync(&v[0], s->kout.alldone, sizeof(int), cudaMemcpyDeviceToHost,
                      s->st) != cudaSuccess ||
      cudaMemcpyAsync(&v[1], s->fault, sizeof(int), cudaMemcpyDeviceToHost, s->st) !=
          cudaSuccess)
    return cuda_check(s, "flag copy");
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return cuda_check(s, "flag sync");
  *out = v[0] || v[1];
  return HZ_OK;
}

bool debug_on() {
  static const bool on = std::getenv("HZ_DEBUG") != nullptr;
  return on;
}

// Opt-in trace (environment HZ_DEBUG=1): Arnoldi state of RHS 0 after a
// Givens step, printed to stderr.  Synchronises the stream.
void debug_trace(hz_solver* s, const KState& ks, const char* label) {
  if (!debug_on()) return;
  cudaStreamSynchronize(s->st);
  int j = 0, done = 0, it = 0;
  double hn = 0, bn = 0;
  cudaMemcpy(&j, ks.jctr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&done, ks.done, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&it, ks.iters, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&hn, ks.hnorm, sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(&bn, ks.bnorm, sizeof(double), cudaMemcpyDeviceToHost);
  const int jj = it > 0 ? it - 1 : 0;
  std::vector<double2> col(jj + 2), g(jj + 2);
  for (int i = 0; i <= jj + 1 && i <= ks.m; ++i)
    cudaMemcpy(&col[i], ks.H + (long long)i * ks.m + jj, sizeof(double2),
               cudaMemcpyDeviceToHost);
  cudaMemcpy(g.data(), ks.g, sizeof(double2) * (jj + 2), cudaMemcpyDeviceToHost);
  fprintf(stderr, "[hz %s] jctr=%d done=%d iters=%d hnorm=%.3e bnorm=%.3e "
          "H[jj][jj]=(%.3e,%.3e) g[jj]=(%.3e,%.3e) g[jj+1]=(%.3e,%.3e) err=%s\n",
          label, j, done, it, hn, bn, col[jj].x, col[jj].y, g[jj].x, g[jj].y,
          g[jj + 1].x, g[jj + 1].y, cudaGetErrorString(cudaGetLastError()));
}

// Event pair around one launch of the profiled kernel class.

// Classical Gram-Schmidt of w against basis columns 0..j with a second pass
// only where the first one cancelled more than a factor 2 (Kahan-Parlett
// "twice is enough": one pass then keeps the basis orthonormal to working
// precision); ||w|| of the result lands in ks.hnorm.
constexpr double kReorthEta = 0.5;

template <class T, class SB>
void cgs2(hz_solver* s, KState& ks, const SB* V, long long vs, long long rs, C<T>* w,
          long long n, int nrhs) {
  cudaStream_t st = s->st;
  KState k = ks;
  k.abytes = nullptr;
  KState kd = k, ka = k;
  if (s->prof_kc == HZ_KC_MDOT) kd.abytes = s->prof_bytes;
  if (s->prof_kc == HZ_KC_MAXPY) ka.abytes = s->prof_bytes;
  for (int pass = 0; pass < 2; ++pass) {
    prof_mark(s, HZ_KC_MDOT);
    launch_mdot<T, SB>(V, vs, rs, w, n, nrhs, kd, pass, st);
    prof_mark(s, HZ_KC_MDOT);
    launch_reduce_cols(k, n, nrhs, pass, st);
    prof_mark(s, HZ_KC_MAXPY);
    launch_maxpy<T, SB>(V, vs, rs, w, n, nrhs, ka, pass, st);
    prof_mark(s, HZ_KC_MAXPY);
    if (pass == 0) launch_reorth_decide(k, n, nrhs, kReorthEta, st);
  }
  launch_reduce_norm(k, n, nrhs, k.hnorm, 1, st);
}

// ------------------------------------------------------------ inner solve
// One Arnoldi step of the inner GMRES: basis vector j (selected on the
// device by the column counter) -> V-cycle -> E -> Gram-Schmidt -> Givens ->
// new basis vector.  Every launch goes to s->st and every argument is fixed
// for the solver, so the step can be captured once and replayed.
// (the part before the Gram-Schmidt step: w = E M_2h^-1 v_j into eb)
template <class T, class SB>
void inner_pre(hz_solver* s, int nrhs) {
  KState& ks = s->kin;
  if (s->d.preconditioner == HZ_PRECOND_TLKM) {
    // TLKM coarse operator: w = R_Z Z M_2h^-1 E v_j
    const long long n1 = s->lv[1].n;
    const long long rs = inner_row(n1);
    const long long vs = (long long)s->d.nrhs_max * rs;
    const LevelDev F = s->lv[0].dev(), Cc = s->lv[1].dev();
    // s->qf holds v_j in compute precision (written with the basis vector)
    apply_E<T>(s, (const C<T>*)s->qf, (C<T>*)s->sb, nrhs, ks.done);
    vcycle<T>(s, 1, vref<T>((C<T>*)s->sb), (C<T>*)s->eb, nrhs, ks.done);
    launch_prolong_z<T>(F, Cc, s->d.bc, s->d.zkind, (const C<T>*)s->eb, (C<T>*)s->q, 0,
                        nrhs, ks.done, s->st);
    launch_restrict_z<T>(F, Cc, s->d.bc, s->d.zkind, vref<T>((C<T>*)s->q), (C<T>*)s->eb,
                         nrhs, ks.done, s->st, rz_scale(s));
    return;
  }
  const long long n1 = s->lv[1].n;
  const long long rs = inner_row(n1);
  const long long vs = (long long)s->d.nrhs_max * rs;
  C<T>* sb = (C<T>*)s->sb;
  // the V-cycle reads the current basis vector: straight from the FP16 basis
  // (inner_in16), or in compute precision from s->qf, where the scaling step
  // left it next to its stored copy
  if constexpr (std::is_same<SB, __half2>::value) {
    if (inner_in16(s)) {
      vcycle_in16(s, 1, vrefe_j<__half2>(s->Qb, ks.jctr, 0, vs), sb, nrhs, ks.done);
      apply_E<T>(s, sb, (C<T>*)s->eb, nrhs, ks.done);
      return;
    }
  }
  vcycle<T>(s, 1, vref<T>(s->qf), sb, nrhs, ks.done);
  apply_E<T>(s, sb, (C<T>*)s->eb, nrhs, ks.done);
}
// (the part after it: Givens update and v_{j+1} = w / ||w||)
template <class T, class SB>
void inner_post(hz_solver* s, int nrhs) {
  KState& ks = s->kin;
  const long long n1 = s->lv[1].n;
  const long long rs = inner_row(n1);
  const long long vs = (long long)s->d.nrhs_max * rs;
  launch_givens(ks, nrhs, s->d.coarse_tol, s->d.coarse_maxit, s->st);
  debug_trace(s, ks, "inner");
  launch_scale_into<T, SB>(vref<T>((C<T>*)s->eb), vrefe_j<SB>((SB*)s->Qb, ks.jctr, 0, vs),
                           rs, ks.hnorm, n1, nrhs, ks.done, s->st,
                           inner_in16(s) ? nullptr : (C<T>*)s->qf);
}
template <class T, class SB>
void inner_step(hz_solver* s, int nrhs) {
  const long long n1 = s->lv[1].n;
  const long long rs = inner_row(n1);
  inner_pre<T, SB>(s, nrhs);
  cgs2<T, SB>(s, s->kin, (SB*)s->Qb, (long long)s->d.nrhs_max * rs, rs, (C<T>*)s->eb, n1,
              nrhs);
  inner_post<T, SB>(s, nrhs);
}

// While s->st is being captured: appends to the graph being captured (the
// outer iteration's, or the body of an enclosing loop) a WHILE node for the
// Krylov loop of deflation level l, whose body is body() plus the loop
// control, preceded by the kernel that sets the loop condition from the
// all-converged flag of ks.  The loop ends when every RHS is done or after
// coarse_maxit iterations (k_givens marks every RHS done at the cap, so the
// count bound is a second guard).  body() may capture the loop of level
// l + 1 inside this body; every body counts only its own kernels
// (body_count_l[l]).
template <class F>
hz_status capture_loop(hz_solver* s, int l, KState& ks, F&& body, int maxit = -1) {
  cudaStream_t st = s->st;
  cudaStream_t cap = l == 1 ? s->cap_body : s->cap_nest[l];
  if (maxit < 0) maxit = s->d.coarse_maxit;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t G = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (!cap || cudaStreamGetCaptureInfo(st, &cs, nullptr, &G, nullptr, nullptr, nullptr) !=
                  cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return cuda_check(s, "loop capture: stream not capturing");
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, G, 0, 0) != cudaSuccess)
    return cuda_check(s, "conditional handle");
  launch_loop_begin(ks.alldone, s->fault, s->loop_it + l, h, st);
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, &G, &deps, nullptr, &nd) !=
      cudaSuccess)
    return cuda_check(s, "capture info");
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, G, deps, nullptr, nd, &p) != cudaSuccess)
    return cuda_check(s, "WHILE node");
  cudaGraph_t body_g = p.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(cap, body_g, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return cuda_check(s, "body capture");
  const long long c0 = launch_counter().load();
  for (int k = l + 1; k < kMaxLevels; ++k) s->body_count_l[k] = 0;
  s->st = cap;
  body();
  launch_loop_next(ks.alldone, s->fault, s->loop_it + l, maxit, s->body_kernels + l, h,
                   s->st);
  s->st = st;
  long long nested = 0;
  for (int k = l + 1; k < kMaxLevels; ++k) nested += s->body_count_l[k];
  s->body_count_l[l] = launch_counter().load() - c0 - nested;
  cudaGraph_t body_out = nullptr;
  if (cudaStreamEndCapture(cap, &body_out) != cudaSuccess)
    return cuda_check(s, "body capture end");
  if (cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies) !=
      cudaSuccess)
    return cuda_check(s, "capture dependencies");
  return cuda_check(s, "loop capture");
}

template <class T, class SB>
hz_status capture_inner_loop(hz_solver* s, int nrhs) {
  return capture_loop(s, 1, s->kin, [&] { inner_step<T, SB>(s, nrhs); });
}

// E v2 = v1 by right-preconditioned GMRES (V-cycle on the coarse CSLP from
// level 1), x0 = 0, stopping at |g_{j+1}| <= coarse_tol ||v1||.
template <class T, class SB>
void coarse_begin(hz_solver* s, const C<T>* v1, int nrhs, const int* done_in) {
  cudaStream_t st = s->st;
  KState& ks = s->kin;
  const long long n1 = s->lv[1].n;
  launch_norm2_part<T>(vref<T>(v1), n1, nrhs, ks, nullptr, st);
  launch_reduce_norm(ks, n1, nrhs, ks.beta, 1, st);
  launch_krylov_init(ks, nrhs, done_in, nullptr, s->d.coarse_tol, st);
  launch_scale_into<T, SB>(vref<T>(v1), vrefe<SB>((SB*)s->Qb), inner_row(n1), ks.hnorm,
                           n1, nrhs, ks.done, st, inner_in16(s) ? nullptr : (C<T>*)s->qf);
}
// x = Q_k y (k the iterations taken), then v2 = M_2h^-1 x (right
// preconditioning)
template <class T, class SB>
void coarse_finish(hz_solver* s, C<T>* v2, int nrhs, const int* done_in) {
  cudaStream_t st = s->st;
  KState& ks = s->kin;
  const long long n1 = s->lv[1].n;
  const long long rs = inner_row(n1);
  launch_trisolve(ks, nrhs, st);
  launch_update<SB, T>((const SB*)s->Qb, (long long)s->d.nrhs_max * rs, rs, ks,
                       (C<T>*)s->eb, 0, n1, nrhs, st);
  if (s->d.preconditioner == HZ_PRECOND_TLKM)   // the operator carries M_2h^-1
    launch_add_conv<T, T>(vref<T>((C<T>*)s->eb), nullptr, vref<T>(v2), n1, nrhs, done_in,
                          st);
  else
    vcycle<T>(s, 1, vref<T>((C<T>*)s->eb), v2, nrhs, done_in);
  launch_accum_iters(ks.iters, s->in_total, s->in_max, nrhs, done_in, st);
}

// ------------------------------------------------------------ multilevel
// Multilevel deflation (deflation_levels = D >= 2; the multilevel direction
// of Sec. 1 / Sec. 7, our reading): the coarse system of level l < D is
// solved by flexible GMRES right-preconditioned by A-DEF1 built from it,
// z = M_l^-1 (v - E_l q) + q, q = Z_l E_{l+1}^-1 R_l v, with the same solve
// one level down inside; level D by GMRES right-preconditioned by the
// V-cycle from level D.  Every level stops at the coarse tolerance.

// E_l x: the chosen coarse operator at level 1, ReD-Glk2 below it (the
// re-discretisation Sec. 5.2.4 suggests for a multilevel method)
template <class T>
void apply_El(hz_solver* s, int l, const C<T>* x, C<T>* y, int nrhs, const int* done) {
  if (l == 1)
    apply_E<T>(s, x, y, nrhs, done);
  else
    launch_glk<T>(s->lv[l].dev(), s->d.bc, 2, x, y, nrhs, done, s->st);
}

// Krylov state, basis and vectors of deflation level l
struct MLView {
  KState* ks;
  void *Q, *qf, *sb, *eb;
};
MLView ml_view(hz_solver* s, int l) {
  if (l == 1) return MLView{&s->kin, s->Qb, s->qf, s->sb, s->eb};
  hz_solver::DefLevel& D = s->dl[l];
  return MLView{&D.ks, D.Q, D.qf, D.sb, D.eb};
}

template <class T, class SB>
hz_status ml_solve(hz_solver* s, int l, const C<T>* v1, C<T>* v2, int nrhs,
                   const int* done_in);

// One Arnoldi step at level l (basis vector j in compute precision in qf):
// z_j = P_l v_j above the deepest level (its directions kept in Zb), the
// V-cycle from level l at the deepest one; w = E_l z_j, Gram-Schmidt,
// Givens, v_{j+1}.  Every launch reads s->st when it is issued: a nested
// loop captured inside switches it and restores it.
template <class T, class SB>
hz_status ml_step(hz_solver* s, int l, int nrhs) {
  const MLView V = ml_view(s, l);
  KState& ks = *V.ks;
  const int bc = s->d.bc, zk = s->d.zkind;
  const long long nl = s->lv[l].n, rs = inner_row(nl);
  const long long vs = (long long)s->d.nrhs_max * rs;
  C<T>* qf = (C<T>*)V.qf;
  C<T>* sb = (C<T>*)V.sb;
  C<T>* eb = (C<T>*)V.eb;
  if (l < s->D) {
    hz_solver::DefLevel& D = s->dl[l];
    hz_solver::DefLevel& Dn = s->dl[l + 1];
    const LevelDev Lf = s->lv[l].dev(), Lc = s->lv[l + 1].dev();
    const long long zs = (long long)s->d.nrhs_max * nl;
    launch_restrict_z<T>(Lf, Lc, bc, zk, vref<T>(qf), (C<T>*)Dn.v1, nrhs, ks.done, s->st);
    const hz_status e =
        ml_solve<T, C<T>>(s, l + 1, (const C<T>*)Dn.v1, (C<T>*)Dn.v2, nrhs, ks.done);
    if (e != HZ_OK) return e;
    launch_prolong_z<T>(Lf, Lc, bc, zk, (const C<T>*)Dn.v2, (C<T>*)D.q, 0, nrhs, ks.done,
                        s->st);
    apply_El<T>(s, l, (const C<T>*)D.q, (C<T>*)D.u, nrhs, ks.done);
    launch_sub<T>(qf, (const C<T>*)D.u, (C<T>*)D.u, nl, nrhs, ks.done, s->st);
    vcycle<T>(s, l, vref<T>((C<T>*)D.u), sb, nrhs, ks.done);
    launch_add_conv<T, T>(vref<T>(sb), (const C<T>*)D.q, vref<T>((C<T>*)D.zj), nl, nrhs,
                          ks.done, s->st);
    launch_add_conv<T, T>(vref<T>((C<T>*)D.zj), nullptr,
                          vref_j<T>((C<T>*)D.Zb, ks.jctr, 0, zs), nl, nrhs, ks.done, s->st);
    apply_El<T>(s, l, (const C<T>*)D.zj, eb, nrhs, ks.done);
  } else {
    vcycle<T>(s, l, vref<T>(qf), sb, nrhs, ks.done);
    apply_El<T>(s, l, sb, eb, nrhs, ks.done);
  }
  cgs2<T, SB>(s, ks, (const SB*)V.Q, vs, rs, eb, nl, nrhs);
  launch_givens(ks, nrhs, s->d.coarse_tol, s->d.coarse_maxit, s->st);
  debug_trace(s, ks, "multilevel");
  launch_scale_into<T, SB>(vref<T>(eb), vrefe_j<SB>((SB*)V.Q, ks.jctr, 0, vs), rs, ks.hnorm,
                           nl, nrhs, ks.done, s->st, qf);
  return cuda_check(s, "multilevel step");
}

// E_l v2 = v1 at deflation level l, x0 = 0; RHS done in the caller
// (done_in) are skipped.  Under capture the loop becomes a WHILE node
// (nested in the enclosing level's body), else it runs on the host with a
// completion check every check_every iterations.
template <class T, class SB>
hz_status ml_solve(hz_solver* s, int l, const C<T>* v1, C<T>* v2, int nrhs,
                   const int* done_in) {
  const MLView V = ml_view(s, l);
  KState& ks = *V.ks;
  const long long nl = s->lv[l].n, rs = inner_row(nl);
  const long long vs = (long long)s->d.nrhs_max * rs;
  const int m = s->d.coarse_maxit;
  launch_norm2_part<T>(vref<T>(v1), nl, nrhs, ks, nullptr, s->st);
  launch_reduce_norm(ks, nl, nrhs, ks.beta, 1, s->st);
  launch_krylov_init(ks, nrhs, done_in, nullptr, s->d.coarse_tol, s->st);
  launch_scale_into<T, SB>(vref<T>(v1), vrefe<SB>((SB*)V.Q), rs, ks.hnorm, nl, nrhs, ks.done,
                           s->st, (C<T>*)V.qf);
  if (s->capturing) {
    hz_status e = HZ_OK;
    const hz_status ce = capture_loop(s, l, ks, [&] { e = ml_step<T, SB>(s, l, nrhs); });
    if (ce != HZ_OK) return ce;
    if (e != HZ_OK) return e;
  } else {
    int all = 0;
    for (int it = 0; it < m; ++it) {
      hz_status e = ml_step<T, SB>(s, l, nrhs);
      if (e != HZ_OK) return e;
      if ((it + 1) % s->check_every == 0 || it + 1 == m) {
        e = read_flag(s, ks.alldone, &all);
        if (e != HZ_OK) return e;
        if (all) break;
      }
    }
  }
  launch_trisolve(ks, nrhs, s->st);
  if (l < s->D) {
    launch_update<C<T>, T>((const C<T>*)s->dl[l].Zb, (long long)s->d.nrhs_max * nl, nl, ks,
                           v2, 0, nl, nrhs, s->st);
  } else {
    launch_update<SB, T>((const SB*)V.Q, vs, rs, ks, (C<T>*)V.eb, 0, nl, nrhs, s->st);
    vcycle<T>(s, l, vref<T>((C<T>*)V.eb), v2, nrhs, done_in);
  }
  if (l == 1) launch_accum_iters(ks.iters, s->in_total, s->in_max, nrhs, done_in, s->st);
  return cuda_check(s, "multilevel coarse solve");
}

template <class T, class SB>
hz_status coarse_solve_sb(hz_solver* s, const C<T>* v1, C<T>* v2, int nrhs,
                          const int* done_in) {
  if (s->ml) return ml_solve<T, SB>(s, 1, v1, v2, nrhs, done_in);
  KState& ks = s->kin;
  const int m = s->d.coarse_maxit;
  coarse_begin<T, SB>(s, v1, nrhs, done_in);
  if (s->capturing) {
    const hz_status e = capture_inner_loop<T, SB>(s, nrhs);
    if (e != HZ_OK) return e;
  } else {
    int all = 0;
    for (int it = 0; it < m; ++it) {
      inner_step<T, SB>(s, nrhs);
      if ((it + 1) % s->check_every == 0 || it + 1 == m) {
        const hz_status e = read_flag(s, ks.alldone, &all);
        if (e != HZ_OK) return e;
        if (all) break;
      }
    }
  }
  coarse_finish<T, SB>(s, v2, nrhs, done_in);
  return cuda_check(s, "coarse solve");
}

template <class T>
hz_status coarse_solve(hz_solver* s, const C<T>* v1, C<T>* v2, int nrhs,
                       const int* done_in) {
  if constexpr (std::is_same<T, float>::value) {
    if (s->basis16) return coarse_solve_sb<T, __half2>(s, v1, v2, nrhs, done_in);
  }
  return coarse_solve_sb<T, C<T>>(s, v1, v2, nrhs, done_in);
}

// ------------------------------------------------------------ A-DEF1
// z = M^-1 (v - A q) + q, q = Z E^-1 R v; v, z FP64 (possibly indexed by the
// outer Arnoldi counter), the preconditioner in precision T.
// (first part: v in precision T, and v1 = R_Z v with deflation)
template <class T>
VRef<T> precond_begin(hz_solver* s, VRef<double> vin, int nrhs, const int* done) {
  const long long n0 = s->lv[0].n;
  VRef<T> v;
  if constexpr (std::is_same<T, double>::value) {
    v = vin;
  } else {
    launch_add_conv<double, T>(vin, nullptr, vref<T>(s->vin), n0, nrhs, done, s->st);
    v = vref<T>(s->vin);
  }
  if (s->d.zkind != HZ_Z_NONE)
    launch_restrict_z<T>(s->lv[0].dev(), s->lv[1].dev(), s->d.bc, s->d.zkind, v,
                         (C<T>*)s->v1, nrhs, done, s->st, rz_scale(s));
  return v;
}
// (last part, after v2 = E^-1 v1: q = Z v2, z = M^-1 (v - A q) + q)
template <class T>
void precond_finish(hz_solver* s, VRef<T> v, VRef<double> zout, int nrhs,
                    const int* done) {
  cudaStream_t st = s->st;
  const int bc = s->d.bc;
  const long long n0 = s->lv[0].n;
  C<T>* yv = (C<T>*)s->yv;
  if (s->d.zkind == HZ_Z_NONE) {
    vcycle<T>(s, 0, v, yv, nrhs, done);
    launch_add_conv<T, double>(vref<T>(yv), nullptr, zout, n0, nrhs, done, st);
    return;
  }
  const LevelDev F = s->lv[0].dev(), Cc = s->lv[1].dev();
  launch_prolong_z<T>(F, Cc, bc, s->d.zkind, (const C<T>*)s->v2, (C<T>*)s->q, 0, nrhs,
                      done, st);
  launch_helm<T>(F, bc, helm1(), vref<T>(s->q), v, (C<T>*)s->t, nrhs, done, st);
  vcycle<T>(s, 0, vref<T>(s->t), yv, nrhs, done);
  launch_add_conv<T, double>(vref<T>(yv), (const C<T>*)s->q, zout, n0, nrhs, done, st);
}

// Practical TLKM (Sec. 3.2.2): w = M^-1 v, v2 from the TLKM coarse system
// with right-hand side R_Z w, q = Z v2, z = w - M^-1 (A q) + q (gamma = 1).
template <class T>
hz_status precond_tlkm(hz_solver* s, VRef<double> vin, VRef<double> zout, int nrhs,
                       const int* done) {
  cudaStream_t st = s->st;
  const int bc = s->d.bc;
  const long long n0 = s->lv[0].n;
  VRef<T> v;
  if constexpr (std::is_same<T, double>::value) {
    v = vin;
  } else {
    launch_add_conv<double, T>(vin, nullptr, vref<T>(s->vin), n0, nrhs, done, st);
    v = vref<T>(s->vin);
  }
  const LevelDev F = s->lv[0].dev(), Cc = s->lv[1].dev();
  C<T>* w = (C<T>*)s->yv;
  vcycle<T>(s, 0, v, w, nrhs, done);
  launch_restrict_z<T>(F, Cc, bc, s->d.zkind, vref<T>(w), (C<T>*)s->v1, nrhs, done, st,
                       rz_scale(s));
  const hz_status e = coarse_solve<T>(s, (const C<T>*)s->v1, (C<T>*)s->v2, nrhs, done);
  if (e != HZ_OK) return e;
  launch_prolong_z<T>(F, Cc, bc, s->d.zkind, (const C<T>*)s->v2, (C<T>*)s->q, 0, nrhs,
                      done, st);
  launch_helm<T>(F, bc, helm1(), vref<T>(s->q), vref<T>(nullptr), (C<T>*)s->t, nrhs,
                 done, st);
  vcycle<T>(s, 0, vref<T>(s->t), (C<T>*)s->fz1, nrhs, done);
  launch_sub_add_widen<T>(w, (const C<T>*)s->fz1, (const C<T>*)s->q, zout, n0, nrhs, done,
                          st);
  return cuda_check(s, "tlkm");
}

template <class T>
hz_status precond(hz_solver* s, VRef<double> vin, VRef<double> zout, int nrhs,
                  const int* done) {
  if (s->d.preconditioner == HZ_PRECOND_TLKM)
    return precond_tlkm<T>(s, vin, zout, nrhs, done);
  const VRef<T> v = precond_begin<T>(s, vin, nrhs, done);
  if (s->d.zkind != HZ_Z_NONE) {
    const hz_status e = coarse_solve<T>(s, (const C<T>*)s->v1, (C<T>*)s->v2, nrhs, done);
    if (e != HZ_OK) return e;
  }
  precond_finish<T>(s, v, zout, nrhs, done);
  return cuda_check(s, "precond");
}

hz_status precond_any(hz_solver* s, VRef<double> v, VRef<double> z, int nrhs,
                      const int* done) {
  return s->mixed ? precond<float>(s, v, z, nrhs, done)
                  : precond<double>(s, v, z, nrhs, done);
}

// ------------------------------------------------------------ outer FGMRES
// One outer FGMRES iteration: z_j = P v_j (A-DEF1), w = A z_j, Gram-Schmidt,
// Givens, v_{j+1}.  Column j is selected on the device.
hz_status outer_step(hz_solver* s, int nrhs, double tol) {
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const long long n0 = s->lv[0].n;
  const long long vs = (long long)s->d.nrhs_max * n0;
  const LevelDev F = dev64(s, 0);
  hz_status e = precond_any(s, vref_j<double>(s->Vo, ko.jctr, 0, vs),
                            vref_j<double>(s->Zo, ko.jctr, 0, vs), nrhs, ko.done);
  if (e != HZ_OK) return e;
  launch_helm<double>(F, s->d.bc, helm1(), vref_j<double>(s->Zo, ko.jctr, 0, vs),
                      vref<double>(nullptr), s->wo, nrhs, ko.done, st);
  cgs2<double, double2>(s, ko, s->Vo, vs, n0, s->wo, n0, nrhs);
  launch_givens(ko, nrhs, tol, s->d.outer_maxit, st);
  debug_trace(s, ko, "outer");
  launch_scale_into<double, double2>(vref<double>(s->wo),
                                    vref_j<double>(s->Vo, ko.jctr, 0, vs), n0,
                                    ko.hnorm, n0, nrhs, ko.done, st);
  return cuda_check(s, "outer step");
}

std::atomic<bool> g_graph_launched{false};
constexpr size_t kMaxGraphs = 4;
constexpr size_t kMaxGcrGraphs = 128;   // one per GCR step

void end_failed_capture(hz_solver* s) {
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  for (int l = kMaxLevels - 1; l >= 0; --l)
    if (s->cap_nest[l] && cudaStreamIsCapturing(s->cap_nest[l], &cs) == cudaSuccess &&
        cs != cudaStreamCaptureStatusNone) {
      cudaStreamEndCapture(s->cap_nest[l], &g);
      g = nullptr;
    }
  if (s->cap_body && cudaStreamIsCapturing(s->cap_body, &cs) == cudaSuccess &&
      cs != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(s->cap_body, &g);
    g = nullptr;
  }
  if (s->cap_main && cudaStreamIsCapturing(s->cap_main, &cs) == cudaSuccess &&
      cs != cudaStreamCaptureStatusNone) {
    if (cudaStreamEndCapture(s->cap_main, &g) == cudaSuccess && g)
      cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

// The instantiated graph of one outer iteration for (nrhs, tol, step),
// captured on first use from issue() (outer_step for FGMRES, step -1; GCR
// step k).  Returns nullptr (with s->err set) if capture or instantiation
// fails.
template <class F>
hz_solver::OuterGraph* outer_graph(hz_solver* s, int nrhs, double tol, int step,
                                   F&& issue) {
  for (hz_solver::OuterGraph& g : s->graphs)
    if (g.nrhs == nrhs && g.tol == tol && g.step == step) return &g;
  const size_t cap = s->d.outer_solver == HZ_OUTER_GCR ? kMaxGcrGraphs : kMaxGraphs;
  if (s->graphs.size() >= cap) {
    cudaStreamSynchronize(s->st);
    cudaGraphExecDestroy(s->graphs.front().ex);
    cudaGraphDestroy(s->graphs.front().g);
    s->graphs.erase(s->graphs.begin());
  }
  bool ok = (s->cap_main ||
             cudaStreamCreateWithFlags(&s->cap_main, cudaStreamNonBlocking) == cudaSuccess) &&
            (s->cap_body ||
             cudaStreamCreateWithFlags(&s->cap_body, cudaStreamNonBlocking) == cudaSuccess);
  for (int l = 2; ok && l <= s->D; ++l)
    ok = s->cap_nest[l] ||
         cudaStreamCreateWithFlags(&s->cap_nest[l], cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cuda_check(s, "capture streams");
    return nullptr;
  }
  cudaStream_t st0 = s->st;
  const long long c0 = launch_counter().load(), h0 = host_op_counter().load();
  if (cudaStreamBeginCapture(s->cap_main, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cuda_check(s, "begin capture");
    return nullptr;
  }
  s->st = s->cap_main;
  s->capturing = true;
  for (long long& c : s->body_count_l) c = 0;
  hz_status e = issue();
  s->body_count = 0;
  for (long long c : s->body_count_l) s->body_count += c;
  s->capturing = false;
  s->st = st0;
  const long long captured = launch_counter().load() - c0;
  launch_counter().fetch_sub(captured);   // nothing ran yet
  host_op_counter().fetch_sub(host_op_counter().load() - h0);
  if (e != HZ_OK) {
    const std::string why = s->err;
    end_failed_capture(s);
    s->err = why;
    return nullptr;
  }
  hz_solver::OuterGraph og{nrhs, tol, step, nullptr, nullptr, captured - s->body_count};
  if (cudaStreamEndCapture(s->cap_main, &og.g) != cudaSuccess) {
    cuda_check(s, "end capture");
    end_failed_capture(s);
    return nullptr;
  }
  if (cudaGraphInstantiate(&og.ex, og.g, 0) != cudaSuccess) {
    cuda_check(s, "graph instantiate");
    cudaGraphDestroy(og.g);
    return nullptr;
  }
  // (level 0, the outer loop of hz_solve_async's graphs, is not captured here)
  for (int l = 1; l < kMaxLevels; ++l) s->body_kernels_host[l] = (int)s->body_count_l[l];
  if (cudaMemcpyAsync(s->body_kernels + 1, s->body_kernels_host + 1,
                      sizeof(int) * (kMaxLevels - 1), cudaMemcpyHostToDevice,
                      st0) != cudaSuccess ||
      cudaStreamSynchronize(st0) != cudaSuccess) {
    cuda_check(s, "graph counter");
    cudaGraphExecDestroy(og.ex);
    cudaGraphDestroy(og.g);
    return nullptr;
  }
  s->graphs.push_back(og);
  return &s->graphs.back();
}

// Outer FGMRES start: ||b||, r0 = b - A x0 (or b), Krylov state, v_0.
hz_status outer_begin(hz_solver* s, const double2* b, double2* x, int nrhs, double tol,
                      int use_x0) {
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const long long n0 = s->lv[0].n;
  const int bc = s->d.bc;
  const LevelDev F = dev64(s, 0);
  cudaMemsetAsync(s->in_total, 0, sizeof(int) * nrhs, st);
  cudaMemsetAsync(s->in_max, 0, sizeof(int) * nrhs, st);
  cudaMemsetAsync(s->out_total, 0, sizeof(int) * nrhs, st);
  // ||b|| over the unknowns (Dirichlet boundary entries of b are ignored)
  launch_add_conv<double, double>(vref<double>(b), nullptr, vref<double>(s->wo), n0,
                                  nrhs, nullptr, st);
  launch_mask_dirichlet<double>(F, bc, s->wo, nrhs, st);
  launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  launch_reduce_norm(ko, n0, nrhs, s->bnorm_o, 1, st);
  if (use_x0) {
    launch_mask_dirichlet<double>(F, bc, x, nrhs, st);
    launch_helm<double>(F, bc, helm1(), vref<double>(x), vref<double>(b), s->wo,
                        nrhs, nullptr, st);
  } else {
    cudaMemsetAsync(x, 0, sizeof(double2) * n0 * nrhs, st);
  }
  launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  launch_reduce_norm(ko, n0, nrhs, ko.beta, 1, st);
  launch_krylov_init(ko, nrhs, nullptr, s->bnorm_o, tol, st);
  launch_scale_into<double, double2>(vref<double>(s->wo), vref<double>(s->Vo), n0,
                                    ko.hnorm, n0, nrhs, ko.done, st);
  return cuda_check(s, "outer init");
}

// The true residual b - A x and the per-RHS report of an outer solve.
hz_status outer_report(hz_solver* s, const double2* b, double2* x, int nrhs,
                       hz_solve_info* info) {
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const long long n0 = s->lv[0].n;
  const int bc = s->d.bc;
  const LevelDev F = dev64(s, 0);
  hz_status e = HZ_OK;
  // true residual
  launch_helm<double>(F, bc, helm1(), vref<double>(x), vref<double>(b), s->wo, nrhs,
                      nullptr, st);
  launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  launch_reduce_norm(ko, n0, nrhs, s->relres, 1, st);
  e = cuda_check(s, "outer finish");
  if (e != HZ_OK) return e;
  std::vector<int> it(nrhs), stt(nrhs), itot(nrhs), imax(nrhs);
  std::vector<double> rr(nrhs), bn(nrhs);
  int fault = 0;
  cudaMemcpyAsync(&fault, s->fault, sizeof(int), cudaMemcpyDeviceToHost, st);
  std::vector<int> otot(nrhs);
  cudaMemcpyAsync(it.data(), ko.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(otot.data(), s->out_total, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(stt.data(), ko.stat, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(itot.data(), s->in_total, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(imax.data(), s->in_max, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(rr.data(), s->relres, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(bn.data(), s->bnorm_o, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(s, "outer sync");
  if (fault) {
    set_err(s, "a Krylov kernel gave up waiting for its staged basis rows");
    cudaMemsetAsync(s->fault, 0, sizeof(int), st);
    return HZ_TIMEOUT;
  }
  hz_status worst = HZ_OK;
  for (int r = 0; r < nrhs; ++r) {
    it[r] += otot[r];
    hz_status sr = (hz_status)stt[r];
    const double rel = bn[r] > 0 ? rr[r] / bn[r] : 0.0;
    if (sr == HZ_OK && !std::isfinite(rel)) sr = HZ_NAN;
    if (info) {
      info[r].outer_iters = it[r];
      info[r].inner_iters_total = itot[r];
      info[r].inner_iters_max = imax[r];
      info[r].relres = rel;
      info[r].status = sr;
    }
    if (worst == HZ_OK && sr != HZ_OK) worst = sr;
  }
  return worst;
}

// ------------------------------------------------------------ autotuning
// Mean ms of `reps` calls of f() on the solver's stream (after one warm-up).
template <class F>
double time_ms(hz_solver* s, int reps, F&& f) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f();
  cudaEventRecord(e0, s->st);
  for (int k = 0; k < reps; ++k) f();
  cudaEventRecord(e1, s->st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)ms / reps;
}

// One launch of the Gram-Schmidt dot (upd = false) or update kernel of the
// inner solver at column j on synthetic basis rows (of the outer solver
// when there is no deflation), with the given kernel variant.
template <class T, class SB>
double time_cgs(hz_solver* s, int nrhs, bool upd, int variant) {
  const bool inner = s->d.zkind != HZ_Z_NONE;
  KState& ks = inner ? s->kin : s->kout;
  const long long n = inner ? s->lv[1].n : s->lv[0].n;
  const long long rs = inner ? inner_row(n) : n;
  const long long vs = (long long)s->d.nrhs_max * rs;
  const int m = inner ? s->d.coarse_maxit : s->d.outer_maxit;
  const int j = m - 1 < 64 ? m - 1 : 64;
  SB* V = inner ? (SB*)s->Qb : (SB*)s->Vo;
  C<T>* w = inner ? (C<T>*)s->eb : (C<T>*)s->wo;
  launch_tune_fill<SB>(V, vs * (j + 1), 0x9e3779b9u, s->st);
  launch_tune_fill<C<T>>(w, n * nrhs, 0x85ebca6bu, s->st);
  launch_tune_state(ks, nrhs, j, s->st);
  // the update's coefficients: a first dot pass
  launch_mdot<T, SB>(V, vs, rs, w, n, nrhs, ks, 0, s->st);
  launch_reduce_cols(ks, n, nrhs, 0, s->st);
  KState k = ks;
  k.abytes = nullptr;
  (upd ? k.updk : k.dotk) = variant;
  return time_ms(s, 5, [&]() {
    if (upd)
      launch_maxpy<T, SB>(V, vs, rs, w, n, nrhs, k, 0, s->st);
    else
      launch_mdot<T, SB>(V, vs, rs, w, n, nrhs, k, 0, s->st);
  });
}

double time_cgs_any(hz_solver* s, int nrhs, bool upd, int variant) {
  if (s->d.zkind == HZ_Z_NONE || !s->mixed)
    return time_cgs<double, double2>(s, nrhs, upd, variant);
  if (s->basis16) return time_cgs<float, __half2>(s, nrhs, upd, variant);
  return time_cgs<float, float2>(s, nrhs, upd, variant);
}

// One V-cycle from level 1 (level 0 without deflation) on synthetic data.
template <class T>
double time_vcycle(hz_solver* s, int nrhs, int fused, int rpb = 0, int tile = 0) {
  const hz_tuning saved = s->tune;
  s->tune.vcycle_fused = fused;
  s->tune.vcycle_rhs_per_block = rpb;
  s->tune.vcycle_tile = tile;
  const int l0 = (s->d.zkind != HZ_Z_NONE && s->L >= 1) ? 1 : 0;
  const long long n = s->lv[l0].n;
  C<T>* in = (C<T>*)(l0 == 1 ? s->sb : s->t);
  C<T>* out = (C<T>*)(l0 == 1 ? s->eb : s->yv);
  launch_tune_fill<C<T>>(in, n * nrhs, 0x165667b1u, s->st);
  const double ms =
      time_ms(s, 5, [&]() { vcycle<T>(s, l0, vref<T>(in), out, nrhs, nullptr); });
  s->tune = saved;
  return ms;
}

template <class T>
double time_e(hz_solver* s, int nrhs, int apply, int rpb, int pairs) {
  const hz_tuning saved = s->tune;
  s->tune.galerkin_apply = apply;
  s->tune.e_rhs_per_block = rpb;
  s->tune.e_column_pairs = pairs;
  const long long n1 = s->lv[1].n;
  launch_tune_fill<C<T>>((C<T>*)s->sb, n1 * nrhs, 0x27d4eb2fu, s->st);
  const double ms = time_ms(s, 8, [&]() {
    apply_E<T>(s, (const C<T>*)s->sb, (C<T>*)s->eb, nrhs, nullptr);
  });
  s->tune = saved;
  return ms;
}

// HZ_TIMEOUT (and the flag cleared) if a Krylov kernel's bounded wait ran out.
hz_status take_fault(hz_solver* s) {
  int f = 0;
  const hz_status e = read_flag(s, s->fault, &f);
  if (e != HZ_OK) return e;
  if (!f) return HZ_OK;
  set_err(s, "a Krylov kernel gave up waiting for its staged basis rows");
  cudaMemsetAsync(s->fault, 0, sizeof(int), s->st);
  return HZ_TIMEOUT;
}

// Outer FGMRES end: x += Z_k y, then the report.
hz_status outer_end(hz_solver* s, const double2* b, double2* x, int nrhs,
                    hz_solve_info* info) {
  const long long n0 = s->lv[0].n;
  launch_trisolve(s->kout, nrhs, s->st);
  launch_update<double2, double>(s->Zo, (long long)s->d.nrhs_max * n0, n0, s->kout, x, 1,
                                 n0, nrhs, s->st);
  return outer_report(s, b, x, nrhs, info);
}

// Flexible GCR as the outer iteration (Sec. 6.3), right-preconditioned by
// A-DEF1.  Step k: u_k = P r (stored in Z slot k), c = A u_k made orthogonal
// to c_0 .. c_{k-1} (V slots) by the same two-pass classical Gram-Schmidt as
// FGMRES, with the coefficients also applied to u_k; both normalised by
// ||c||; then x += (c_k, r) u_k, r -= (c_k, r) c_k.  Issued eagerly.
// One GCR step k on the solver's own iterate xg and residual ro; every
// argument is fixed for (nrhs, tol, k), so the step can be captured.
hz_status gcr_step(hz_solver* s, int nrhs, double tol, int k) {
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const long long n0 = s->lv[0].n;
  const long long vs = (long long)s->d.nrhs_max * n0;
  const int m = s->d.outer_maxit;
  KState kg = ko;      // the dot (c_k, r): one basis vector
  kg.jctr = s->izero;
  kg.abytes = nullptr;
  double2* u = s->Zo + k * vs;
  double2* c = s->Vo + k * vs;
  hz_status e = precond_any(s, vref<double>(s->ro), vref<double>(u), nrhs, ko.done);
  if (e != HZ_OK) return e;
  st = s->st;
  launch_helm<double>(dev64(s, 0), s->d.bc, helm1(), vref<double>(u), vref<double>(nullptr),
                      s->wo, nrhs, ko.done, st);
  if (k > 0) {
    launch_fill_int(ko.jctr, k - 1, 1, st);
    for (int pass = 0; pass < 2; ++pass) {
      launch_mdot<double, double2>(s->Vo, vs, n0, s->wo, n0, nrhs, ko, pass, st);
      launch_reduce_cols(ko, n0, nrhs, pass, st);
      // the directions first: the update of c leaves its norm in npart
      launch_maxpy<double, double2>(s->Zo, vs, n0, u, n0, nrhs, ko, pass, st);
      launch_maxpy<double, double2>(s->Vo, vs, n0, s->wo, n0, nrhs, ko, pass, st);
      if (pass == 0) launch_reorth_decide(ko, n0, nrhs, kReorthEta, st);
    }
  } else {
    launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  }
  launch_reduce_norm(ko, n0, nrhs, ko.hnorm, 1, st);
  launch_scale_into<double, double2>(vref<double>(s->wo), vref<double>(c), n0, ko.hnorm, n0,
                                    nrhs, ko.done, st);
  launch_scale_into<double, double2>(vref<double>(u), vref<double>(u), n0, ko.hnorm, n0,
                                    nrhs, ko.done, st);
  launch_mdot<double, double2>(c, vs, n0, s->ro, n0, nrhs, kg, 0, st);
  launch_reduce_cols(kg, n0, nrhs, 0, st);
  launch_gcr_update(s->xg, s->ro, u, c, n0, nrhs, ko, st);
  launch_reduce_norm(ko, n0, nrhs, ko.beta, 1, st);
  launch_gcr_check(ko, ko.beta, nrhs, tol, k, m, st);
  return cuda_check(s, "gcr step");
}

// Flexible GCR as the outer iteration (Sec. 6.3), right-preconditioned by
// A-DEF1.  Step k: u_k = P r (stored in Z slot k), c = A u_k made orthogonal
// to c_0 .. c_{k-1} (V slots) by the same two-pass classical Gram-Schmidt as
// FGMRES, with the coefficients also applied to u_k; both normalised by
// ||c||; then x += (c_k, r) u_k, r -= (c_k, r) c_k.  Each step runs as a
// CUDA graph of its own (captured on first use, one per step index), the
// iterate accumulating in the solver's buffer and copied out at the end.
hz_status solve_gcr(hz_solver* s, const double2* b, double2* x, int nrhs, double tol,
                    int use_x0, hz_solve_info* info) {
  cudaStream_t st = s->st;
  const long long n0 = s->lv[0].n;
  const int m = s->d.outer_maxit;
  hz_status e = outer_begin(s, b, x, nrhs, tol, use_x0);
  if (e != HZ_OK) return e;
  // r = b - A x0, as left in wo by outer_begin; x0 (or 0) into xg
  launch_add_conv<double, double>(vref<double>(s->wo), nullptr, vref<double>(s->ro), n0,
                                  nrhs, nullptr, st);
  launch_add_conv<double, double>(vref<double>(x), nullptr, vref<double>(s->xg), n0, nrhs,
                                  nullptr, st);
  const bool graphs = !s->d.no_cuda_graph && s->prof_kc == HZ_KC_NONE && !debug_on();
  int all = 0;
  e = read_outer_flag(s, &all);
  if (e != HZ_OK) return e;
  for (int k = 0; k < m && !all; ++k) {
    hz_solver::OuterGraph* og = nullptr;
    if (graphs && k < (int)kMaxGcrGraphs) {
      og = outer_graph(s, nrhs, tol, k, [&] { return gcr_step(s, nrhs, tol, k); });
      if (!og) return HZ_CUDA_ERROR;
      if (cudaGraphLaunch(og->ex, st) != cudaSuccess) return cuda_check(s, "graph launch");
      launch_counter().fetch_add(og->kernels);
      host_op_counter().fetch_add(1);
      g_graph_launched.store(true);
    } else {
      e = gcr_step(s, nrhs, tol, k);
      if (e != HZ_OK) return e;
    }
    e = read_outer_flag(s, &all);
    if (e != HZ_OK) return e;
  }
  launch_add_conv<double, double>(vref<double>(s->xg), nullptr, vref<double>(x), n0, nrhs,
                                  nullptr, st);
  return outer_report(s, b, x, nrhs, info);
}

// The per-RHS report of an outer solve written to device memory (the
// device-side counterpart of outer_report; a raised fault flag reports
// HZ_TIMEOUT for every RHS and is cleared).
__global__ void k_solve_info(hz_solve_info* info, KState ko, const int* in_total,
                             const int* in_max, const int* out_total, const double* relres,
                             const double* bnorm, int* fault, int nrhs) {
  const int r = threadIdx.x;
  const int f = *fault;
  __syncthreads();
  if (r < nrhs) {
    hz_status sr = (hz_status)ko.stat[r];
    const double rel = bnorm[r] > 0 ? relres[r] / bnorm[r] : 0.0;
    if (sr == HZ_OK && !isfinite(rel)) sr = HZ_NAN;
    if (f) sr = HZ_TIMEOUT;
    info[r].outer_iters = ko.iters[r] + out_total[r];
    info[r].inner_iters_total = in_total[r];
    info[r].inner_iters_max = in_max[r];
    info[r].relres = rel;
    info[r].status = sr;
  }
  __syncthreads();
  if (r == 0) *fault = 0;
}

// The whole FGMRES solve as one graph (hz_solve_async): start, the outer
// loop as a WHILE node with the inner loop nested in its body, the update
// of x, the true residual and the report kernel.
hz_status capture_solve(hz_solver* s, const double2* b, double2* x, int nrhs, double tol,
                        int use_x0, hz_solve_info* info_dev) {
  const long long n0 = s->lv[0].n;
  KState& ko = s->kout;
  hz_status e = outer_begin(s, b, x, nrhs, tol, use_x0);
  if (e != HZ_OK) return e;
  hz_status es = HZ_OK;
  e = capture_loop(s, 0, ko, [&] { es = outer_step(s, nrhs, tol); }, s->d.outer_maxit);
  if (e != HZ_OK) return e;
  if (es != HZ_OK) return es;
  cudaStream_t st = s->st;
  launch_trisolve(ko, nrhs, st);
  launch_update<double2, double>(s->Zo, (long long)s->d.nrhs_max * n0, n0, ko, x, 1, n0,
                                 nrhs, st);
  launch_helm<double>(dev64(s, 0), s->d.bc, helm1(), vref<double>(x), vref<double>(b),
                      s->wo, nrhs, nullptr, st);
  launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  launch_reduce_norm(ko, n0, nrhs, s->relres, 1, st);
  HZ_COUNT();
  k_solve_info<<<1, 1024, 0, st>>>(info_dev, ko, s->in_total, s->in_max, s->out_total,
                                   s->relres, s->bnorm_o, s->fault, nrhs);
  return cuda_check(s, "solve capture");
}

hz_status solve_async(hz_solver* s, const double2* b, double2* x, int nrhs, double tol,
                      int use_x0, hz_solve_info* info_dev) {
  hz_solver::SolveGraph* sg = nullptr;
  for (hz_solver::SolveGraph& g : s->solve_graphs)
    if (g.nrhs == nrhs && g.tol == tol && g.use_x0 == use_x0 && g.b == b && g.x == x &&
        g.info == info_dev)
      sg = &g;
  if (!sg) {
    if (s->solve_graphs.size() >= kMaxGraphs) {
      cudaStreamSynchronize(s->st);
      cudaGraphExecDestroy(s->solve_graphs.front().ex);
      cudaGraphDestroy(s->solve_graphs.front().g);
      s->solve_graphs.erase(s->solve_graphs.begin());
    }
    bool ok = (s->cap_main ||
               cudaStreamCreateWithFlags(&s->cap_main, cudaStreamNonBlocking) == cudaSuccess) &&
              (s->cap_body ||
               cudaStreamCreateWithFlags(&s->cap_body, cudaStreamNonBlocking) == cudaSuccess);
    for (int l = 0; ok && l <= s->D; ++l)
      if (l != 1)
        ok = s->cap_nest[l] ||
             cudaStreamCreateWithFlags(&s->cap_nest[l], cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) return cuda_check(s, "capture streams");
    cudaStream_t st0 = s->st;
    const long long c0 = launch_counter().load(), h0 = host_op_counter().load();
    if (cudaStreamBeginCapture(s->cap_main, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return cuda_check(s, "begin capture");
    s->st = s->cap_main;
    s->capturing = true;
    for (long long& c : s->body_count_l) c = 0;
    const hz_status e = capture_solve(s, b, x, nrhs, tol, use_x0, info_dev);
    s->capturing = false;
    s->st = st0;
    long long body = 0;
    for (long long c : s->body_count_l) body += c;
    const long long captured = launch_counter().load() - c0;
    launch_counter().fetch_sub(captured);
    host_op_counter().fetch_sub(host_op_counter().load() - h0);
    if (e != HZ_OK) {
      const std::string why = s->err;
      end_failed_capture(s);
      s->err = why;
      return e;
    }
    hz_solver::SolveGraph g{nrhs, use_x0, tol, b, x, info_dev, nullptr, nullptr,
                            captured - body};
    if (cudaStreamEndCapture(s->cap_main, &g.g) != cudaSuccess) {
      const hz_status ce = cuda_check(s, "end capture");
      end_failed_capture(s);
      return ce;
    }
    if (cudaGraphInstantiate(&g.ex, g.g, 0) != cudaSuccess) {
      const hz_status ce = cuda_check(s, "graph instantiate");
      cudaGraphDestroy(g.g);
      return ce;
    }
    for (int l = 0; l < kMaxLevels; ++l) s->body_kernels_host[l] = (int)s->body_count_l[l];
    if (cudaMemcpyAsync(s->body_kernels, s->body_kernels_host, sizeof(int) * kMaxLevels,
                        cudaMemcpyHostToDevice, s->st) != cudaSuccess)
      return cuda_check(s, "graph counter");
    s->solve_graphs.push_back(g);
    sg = &s->solve_graphs.back();
  }
  if (cudaGraphLaunch(sg->ex, s->st) != cudaSuccess) return cuda_check(s, "graph launch");
  launch_counter().fetch_add(sg->kernels);
  host_op_counter().fetch_add(1);
  g_graph_launched.store(true);
  return HZ_OK;
}

// FGMRES restart (hz_desc.restart): x += Z_k y of the finished cycle, its
// iterations added to out_total, then a new Arnoldi start from the true
// residual b - A x with the stopping reference ||b|| kept; RHS that stopped
// stay stopped.
hz_status outer_restart(hz_solver* s, const double2* b, double2* x, int nrhs, double tol) {
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const long long n0 = s->lv[0].n;
  launch_trisolve(ko, nrhs, st);
  launch_update<double2, double>(s->Zo, (long long)s->d.nrhs_max * n0, n0, ko, x, 1, n0,
                                 nrhs, st);
  launch_accum_iters(ko.iters, s->out_total, s->out_max, nrhs, nullptr, st);
  launch_helm<double>(dev64(s, 0), s->d.bc, helm1(), vref<double>(x), vref<double>(b),
                      s->wo, nrhs, nullptr, st);
  launch_norm2_part<double>(vref<double>(s->wo), n0, nrhs, ko, nullptr, st);
  launch_reduce_norm(ko, n0, nrhs, ko.beta, 1, st);
  launch_krylov_init(ko, nrhs, ko.done, s->bnorm_o, tol, st);
  launch_scale_into<double, double2>(vref<double>(s->wo), vref<double>(s->Vo), n0,
                                    ko.hnorm, n0, nrhs, ko.done, st);
  return cuda_check(s, "outer restart");
}

hz_status solve_dev(hz_solver* s, const double2* b, double2* x, int nrhs,
                    double tol, int use_x0, hz_solve_info* info) {
  if (s->d.outer_solver == HZ_OUTER_GCR) return solve_gcr(s, b, x, nrhs, tol, use_x0, info);
  cudaStream_t st = s->st;
  KState& ko = s->kout;
  const int m = s->d.outer_maxit;
  hz_status e = outer_begin(s, b, x, nrhs, tol, use_x0);
  if (e != HZ_OK) return e;
  int all = 0;
  // graphs replay fixed launches: the per-launch events of the profiler
  // and the trace's host reads need the launches issued one by one
  hz_solver::OuterGraph* og = nullptr;
  if (!s->d.no_cuda_graph && s->prof_kc == HZ_KC_NONE && !debug_on()) {
    og = outer_graph(s, nrhs, tol, -1, [&] { return outer_step(s, nrhs, tol); });
    if (!og) return HZ_CUDA_ERROR;
  }
  e = read_outer_flag(s, &all);
  if (e != HZ_OK) return e;
  const int restart = s->d.restart;
  int cycle = 0;
  for (int it = 0; it < m && !all; ++it) {
    if (og) {
      if (cudaGraphLaunch(og->ex, st) != cudaSuccess) return cuda_check(s, "graph launch");
      launch_counter().fetch_add(og->kernels);
      host_op_counter().fetch_add(1);
      g_graph_launched.store(true);
    } else {
      e = outer_step(s, nrhs, tol);
      if (e != HZ_OK) return e;
    }
    e = read_outer_flag(s, &all);
    if (e != HZ_OK) return e;
    if (restart > 0 && ++cycle == restart && !all && it + 1 < m) {
      e = outer_restart(s, b, x, nrhs, tol);
      if (e != HZ_OK) return e;
      cycle = 0;
      e = read_outer_flag(s, &all);
      if (e != HZ_OK) return e;
    }
  }
  return outer_end(s, b, x, nrhs, info);
}

// ------------------------------------------------------------ uneven grids
// Solvers on grids of different sizes advanced together: every Krylov
// iteration of all members runs in lockstep, each member's stencil work is
// launched for its own grid, and the Gram-Schmidt kernels of all members run
// as one persistent launch over a table of their tiles (k_*_group).
struct Member {
  hz_solver* s;
  int nrhs;
};

template <class T, class SB>
void cgs2_group(const std::vector<Member>& M, bool inner, cudaStream_t st) {
  GroupDesc gd{};
  gd.count = (int)M.size();
  long long start = 0;
  for (int g = 0; g < gd.count; ++g) {
    hz_solver* s = M[g].s;
    GroupMember& m = gd.m[g];
    const long long n = inner ? s->lv[1].n : s->lv[0].n;
    m.rs = inner ? inner_row(n) : n;
    m.vstride = (long long)s->d.nrhs_max * m.rs;
    m.V = inner ? s->Qb : (const void*)s->Vo;
    m.w = inner ? s->eb : (void*)s->wo;
    m.n = n;
    m.ks = inner ? s->kin : s->kout;
    m.ks.abytes = nullptr;
    m.nrhs = M[g].nrhs;
    m.nblk = krylov_nblk(n);
    gd.start[g] = start;
    start += (long long)m.nrhs * m.nblk;
  }
  gd.start[gd.count] = start;
  for (int pass = 0; pass < 2; ++pass) {
    launch_mdot_group<T, SB>(gd, pass, st);
    for (int g = 0; g < gd.count; ++g)
      launch_reduce_cols(gd.m[g].ks, gd.m[g].n, gd.m[g].nrhs, pass, st);
    launch_maxpy_group<T, SB>(gd, pass, st);
    if (pass == 0)
      for (int g = 0; g < gd.count; ++g)
        launch_reorth_decide(gd.m[g].ks, gd.m[g].n, gd.m[g].nrhs, kReorthEta, st);
  }
  for (int g = 0; g < gd.count; ++g)
    launch_reduce_norm(gd.m[g].ks, gd.m[g].n, gd.m[g].nrhs, gd.m[g].ks.hnorm, 1, st);
}

// all[g] = the all-converged flag of member g's inner or outer solver
hz_status read_flags(const std::vector<Member>& M, bool inner, std::vector<int>& all,
                     cudaStream_t st) {
  all.assign(M.size(), 0);
  for (size_t g = 0; g < M.size(); ++g)
    cudaMemcpyAsync(&all[g], inner ? M[g].s->kin.alldone : M[g].s->kout.alldone,
                    sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(M[0].s, "group flags");
  return HZ_OK;
}

// A group solve issued as CUDA graphs: one graph per outer iteration of the
// active members (captured on first use for each set of active members and
// destroyed when the call returns).  In it every member's own work (its
// stencil, transfer and E kernels) runs on a branch of its own, so the
// members' grids share the GPU; the branches join before each grouped
// Gram-Schmidt step.  The inner coarse solves advance together in a WHILE
// node that repeats while some member's inner solve is not done.
struct GroupCtx {
  bool capturing = false;
  cudaStream_t main = nullptr;           // stream being captured (outer level)
  cudaStream_t body = nullptr;           // WHILE body capture stream
  std::vector<cudaStream_t> br_out, br_in;   // member branches (outer, body)
  std::vector<cudaEvent_t> ev;           // fork + one join per member
  long long body_count = 0;              // own kernels of the WHILE body
  int* flag = nullptr;                   // device: all members' inner solves done
  int* loop_it = nullptr;                // device: WHILE iterations
  int* body_kernels = nullptr;           // device: body_count
  ~GroupCtx() {
    for (cudaStream_t c : br_out) if (c) cudaStreamDestroy(c);
    for (cudaStream_t c : br_in) if (c) cudaStreamDestroy(c);
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
  }
};

// f(g) for every member g: on its own branch of the captured graph
// (forked from and joined back to st), or in order on st.
template <class F>
void each_member(const std::vector<Member>& M, GroupCtx* gc, bool body, cudaStream_t st,
                 F&& f) {
  if (!gc || !gc->capturing) {
    for (size_t g = 0; g < M.size(); ++g) f(g);
    return;
  }
  const std::vector<cudaStream_t>& br = body ? gc->br_in : gc->br_out;
  cudaEventRecord(gc->ev[0], st);
  for (size_t g = 0; g < M.size(); ++g) {
    cudaStreamWaitEvent(br[g], gc->ev[0], 0);
    M[g].s->st = br[g];
    f(g);
    M[g].s->st = st;
    cudaEventRecord(gc->ev[1 + g], br[g]);
  }
  for (size_t g = 0; g < M.size(); ++g) cudaStreamWaitEvent(st, gc->ev[1 + g], 0);
}

FlagSet inner_flags(const std::vector<Member>& M) {
  FlagSet fs{};
  fs.n = (int)M.size();
  for (size_t g = 0; g < M.size(); ++g) fs.f[g] = M[g].s->kin.alldone;
  return fs;
}

template <class T, class SB>
hz_status coarse_solve_group(const std::vector<Member>& M, cudaStream_t st, GroupCtx* gc) {
  int m = 0;
  for (const Member& g : M) m = g.s->d.coarse_maxit > m ? g.s->d.coarse_maxit : m;
  each_member(M, gc, false, st, [&](size_t g) {
    coarse_begin<T, SB>(M[g].s, (const C<T>*)M[g].s->v1, M[g].nrhs, M[g].s->kout.done);
  });
  if (gc && gc->capturing) {
    // the loop as a WHILE node over all members
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t G = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(st, &cs, nullptr, &G, nullptr, nullptr, nullptr) !=
            cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
      return cuda_check(M[0].s, "group loop capture: stream not capturing");
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, G, 0, 0) != cudaSuccess)
      return cuda_check(M[0].s, "conditional handle");
    launch_all_of(inner_flags(M), gc->flag, st);
    launch_loop_begin(gc->flag, nullptr, gc->loop_it, h, st);
    if (cudaStreamGetCaptureInfo(st, &cs, nullptr, &G, &deps, nullptr, &nd) != cudaSuccess)
      return cuda_check(M[0].s, "capture info");
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, G, deps, nullptr, nd, &p) != cudaSuccess)
      return cuda_check(M[0].s, "WHILE node");
    if (cudaStreamBeginCaptureToGraph(gc->body, p.conditional.phGraph_out[0], nullptr,
                                      nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess)
      return cuda_check(M[0].s, "body capture");
    const long long c0 = launch_counter().load();
    each_member(M, gc, true, gc->body, [&](size_t g) { inner_pre<T, SB>(M[g].s, M[g].nrhs); });
    cgs2_group<T, SB>(M, true, gc->body);
    each_member(M, gc, true, gc->body,
                [&](size_t g) { inner_post<T, SB>(M[g].s, M[g].nrhs); });
    launch_all_of(inner_flags(M), gc->flag, gc->body);
    launch_loop_next(gc->flag, nullptr, gc->loop_it, m, gc->body_kernels, h, gc->body);
    gc->body_count = launch_counter().load() - c0;
    cudaGraph_t bo = nullptr;
    if (cudaStreamEndCapture(gc->body, &bo) != cudaSuccess)
      return cuda_check(M[0].s, "body capture end");
    if (cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
      return cuda_check(M[0].s, "capture dependencies");
  } else {
    const int every = M[0].s->check_every;
    std::vector<int> all;
    for (int it = 0; it < m; ++it) {
      for (const Member& g : M) inner_pre<T, SB>(g.s, g.nrhs);
      cgs2_group<T, SB>(M, true, st);
      for (const Member& g : M) inner_post<T, SB>(g.s, g.nrhs);
      if ((it + 1) % every == 0 || it + 1 == m) {
        const hz_status e = read_flags(M, true, all, st);
        if (e != HZ_OK) return e;
        bool done = true;
        for (int a : all) done = done && a;
        if (done) break;
      }
    }
  }
  each_member(M, gc, false, st, [&](size_t g) {
    coarse_finish<T, SB>(M[g].s, (C<T>*)M[g].s->v2, M[g].nrhs, M[g].s->kout.done);
  });
  return cuda_check(M[0].s, "group coarse solve");
}

template <class T>
hz_status outer_step_group(const std::vector<Member>& M, double tol, cudaStream_t st,
                           GroupCtx* gc) {
  std::vector<VRef<T>> v(M.size());
  each_member(M, gc, false, st, [&](size_t g) {
    hz_solver* s = M[g].s;
    const long long vs = (long long)s->d.nrhs_max * s->lv[0].n;
    v[g] = precond_begin<T>(s, vref_j<double>(s->Vo, s->kout.jctr, 0, vs), M[g].nrhs,
                            s->kout.done);
  });
  if (M[0].s->d.zkind != HZ_Z_NONE) {
    hz_status e;
    if constexpr (std::is_same<T, float>::value) {
      e = M[0].s->basis16 ? coarse_solve_group<T, __half2>(M, st, gc)
                          : coarse_solve_group<T, C<T>>(M, st, gc);
    } else {
      e = coarse_solve_group<T, C<T>>(M, st, gc);
    }
    if (e != HZ_OK) return e;
  }
  each_member(M, gc, false, st, [&](size_t g) {
    hz_solver* s = M[g].s;
    const long long vs = (long long)s->d.nrhs_max * s->lv[0].n;
    precond_finish<T>(s, v[g], vref_j<double>(s->Zo, s->kout.jctr, 0, vs), M[g].nrhs,
                      s->kout.done);
    launch_helm<double>(dev64(s, 0), s->d.bc, helm1(),
                        vref_j<double>(s->Zo, s->kout.jctr, 0, vs), vref<double>(nullptr),
                        s->wo, M[g].nrhs, s->kout.done, s->st);
  });
  cgs2_group<double, double2>(M, false, st);
  each_member(M, gc, false, st, [&](size_t g) {
    hz_solver* s = M[g].s;
    const long long n0 = s->lv[0].n;
    const long long vs = (long long)s->d.nrhs_max * n0;
    launch_givens(s->kout, M[g].nrhs, tol, s->d.outer_maxit, s->st);
    launch_scale_into<double, double2>(vref<double>(s->wo),
                                      vref_j<double>(s->Vo, s->kout.jctr, 0, vs), n0,
                                      s->kout.hnorm, n0, M[g].nrhs, s->kout.done, s->st);
  });
  return cuda_check(M[0].s, "group outer step");
}

struct GroupGraph {
  unsigned mask;
  cudaGraph_t g;
  cudaGraphExec_t ex;
  long long kernels;   // kernels of one launch outside the WHILE body
};

// Captures (or returns the captured) graph of one outer iteration of the
// active members act (bit g of mask = member g active).
GroupGraph* group_graph(const std::vector<Member>& act, unsigned mask, double tol,
                        GroupCtx& gc, std::vector<GroupGraph>& graphs, cudaStream_t st) {
  for (GroupGraph& g : graphs)
    if (g.mask == mask) return &g;
  hz_solver* s0 = act[0].s;
  const long long c0 = launch_counter().load(), h0 = host_op_counter().load();
  if (cudaStreamBeginCapture(gc.main, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cuda_check(s0, "begin group capture");
    return nullptr;
  }
  for (const Member& m : act) m.s->st = gc.main;
  gc.capturing = true;
  gc.body_count = 0;
  const hz_status e = s0->mixed ? outer_step_group<float>(act, tol, gc.main, &gc)
                                : outer_step_group<double>(act, tol, gc.main, &gc);
  gc.capturing = false;
  for (const Member& m : act) m.s->st = st;
  const long long captured = launch_counter().load() - c0;
  launch_counter().fetch_sub(captured);
  host_op_counter().fetch_sub(host_op_counter().load() - h0);
  GroupGraph gg{mask, nullptr, nullptr, captured - gc.body_count};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(gc.body, &cs) == cudaSuccess &&
      cs != cudaStreamCaptureStatusNone) {   // a failure inside the WHILE body
    cudaGraph_t bg = nullptr;
    cudaStreamEndCapture(gc.body, &bg);
  }
  const cudaError_t ce = cudaStreamEndCapture(gc.main, &gg.g);
  if (e != HZ_OK || ce != cudaSuccess) {
    if (ce == cudaSuccess && gg.g) cudaGraphDestroy(gg.g);
    cudaGetLastError();
    if (e == HZ_OK) set_err(s0, "group graph capture failed");
    return nullptr;
  }
  if (cudaGraphInstantiate(&gg.ex, gg.g, 0) != cudaSuccess) {
    cuda_check(s0, "group graph instantiate");
    cudaGraphDestroy(gg.g);
    return nullptr;
  }
  const int bc = (int)gc.body_count;
  if (cudaMemcpyAsync(gc.body_kernels, &bc, sizeof(int), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cuda_check(s0, "group graph counter");
    cudaGraphExecDestroy(gg.ex);
    cudaGraphDestroy(gg.g);
    return nullptr;
  }
  graphs.push_back(gg);
  return &graphs.back();
}

// Member g solves b[g] -> x[g] (x0 = 0); all members already run on st.
hz_status solve_group_dev(const std::vector<Member>& M, const double2* const* b,
                          double2* const* x, double tol, hz_solve_info* const* info,
                          cudaStream_t st) {
  const int K = (int)M.size();
  int m = 0;
  bool graphs_ok = true;
  for (int g = 0; g < K; ++g) {
    const hz_status e = outer_begin(M[g].s, b[g], x[g], M[g].nrhs, tol, 0);
    if (e != HZ_OK) return e;
    m = M[g].s->d.outer_maxit > m ? M[g].s->d.outer_maxit : m;
    graphs_ok = graphs_ok && !M[g].s->d.no_cuda_graph && M[g].s->prof_kc == HZ_KC_NONE;
  }
  graphs_ok = graphs_ok && !debug_on();
  // graph mode: branch streams, fork/join events and the group's device
  // flags (in member 0's workspace)
  GroupCtx gc;
  std::vector<GroupGraph> graphs;
  if (graphs_ok) {
    hz_solver* s0 = M[0].s;
    bool ok = s0->cap_main ||
              cudaStreamCreateWithFlags(&s0->cap_main, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && (s0->cap_body ||
                cudaStreamCreateWithFlags(&s0->cap_body, cudaStreamNonBlocking) == cudaSuccess);
    gc.main = s0->cap_main;
    gc.body = s0->cap_body;
    gc.br_out.assign(K, nullptr);
    gc.br_in.assign(K, nullptr);
    gc.ev.assign(K + 1, nullptr);
    for (int g = 0; ok && g < K; ++g)
      ok = cudaStreamCreateWithFlags(&gc.br_out[g], cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamCreateWithFlags(&gc.br_in[g], cudaStreamNonBlocking) == cudaSuccess;
    for (int g = 0; ok && g <= K; ++g)
      ok = cudaEventCreateWithFlags(&gc.ev[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_check(s0, "group graph streams");
    gc.flag = s0->grp;
    gc.loop_it = s0->grp + 1;
    gc.body_kernels = s0->grp + 2;
  }
  std::vector<int> all;
  hz_status e = read_flags(M, false, all, st);
  if (e != HZ_OK) return e;
  for (int it = 0; it < m; ++it) {
    std::vector<Member> act;
    unsigned mask = 0;
    for (int g = 0; g < K; ++g)
      if (!all[g]) {
        act.push_back(M[g]);
        mask |= 1u << g;
      }
    if (act.empty()) break;
    if (graphs_ok) {
      GroupGraph* gg = group_graph(act, mask, tol, gc, graphs, st);
      if (!gg) {
        e = HZ_CUDA_ERROR;
        break;
      }
      if (cudaGraphLaunch(gg->ex, st) != cudaSuccess) {
        e = cuda_check(M[0].s, "group graph launch");
        break;
      }
      launch_counter().fetch_add(gg->kernels);
      host_op_counter().fetch_add(1);
      g_graph_launched.store(true);
    } else {
      e = M[0].s->mixed ? outer_step_group<float>(act, tol, st, nullptr)
                        : outer_step_group<double>(act, tol, st, nullptr);
      if (e != HZ_OK) break;
    }
    std::vector<int> now;
    e = read_flags(act, false, now, st);
    if (e != HZ_OK) break;
    for (size_t a = 0, g = 0; g < (size_t)K; ++g)
      if (!all[g]) all[g] = now[a++];
  }
  if (!graphs.empty()) cudaStreamSynchronize(st);
  for (GroupGraph& g : graphs) {
    cudaGraphExecDestroy(g.ex);
    cudaGraphDestroy(g.g);
  }
  if (e != HZ_OK) return e;
  hz_status worst = HZ_OK;
  for (int g = 0; g < K; ++g) {
    e = outer_end(M[g].s, b[g], x[g], M[g].nrhs, info ? info[g] : nullptr);
    if (e == HZ_CUDA_ERROR || e == HZ_TIMEOUT) return e;
    if (worst == HZ_OK) worst = e;
  }
  return worst;
}

// Checks a group and runs every member on members[0]'s stream while alive.
struct GroupScope {
  std::vector<hz_solver*> S;
  std::vector<cudaStream_t> saved;
  hz_status status = HZ_OK;
  GroupScope(hz_solver* const* members, int count) {
    if (!members || count < 1 || count > kMaxGroup) {
      status = HZ_INVALID_ARG;
      return;
    }
    for (int g = 0; g < count; ++g) {
      hz_solver* s = members[g];
      if (!s) {
        status = HZ_INVALID_ARG;
        return;
      }
      for (hz_solver* t : S)
        if (t == s) status = HZ_INVALID_ARG;
      if (s->d.outer_solver != HZ_OUTER_FGMRES ||
          s->d.preconditioner != HZ_PRECOND_ADEF1 || s->ml) {
        set_err(s, "group solves use flexible GMRES members with A-DEF1");
        status = HZ_INVALID_ARG;
      }
      if (g > 0 && (s->mixed != S[0]->mixed || s->basis16 != S[0]->basis16 ||
                    (s->d.zkind == HZ_Z_NONE) != (S[0]->d.zkind == HZ_Z_NONE))) {
        set_err(S[0], "group members differ in precision, inner-basis storage or "
                      "deflation");
        status = HZ_INVALID_ARG;
      }
      S.push_back(s);
    }
    if (status != HZ_OK) return;
    for (hz_solver* s : S) {
      saved.push_back(s->st);
      s->st = S[0]->st;
    }
  }
  ~GroupScope() {
    for (size_t g = 0; g < saved.size(); ++g) S[g]->st = saved[g];
  }
};

template <class T>
hz_status apply_op(hz_solver* s, hz_op op, int level, const double2* x, double2* y,
                   int nrhs) {
  cudaStream_t st = s->st;
  const int bc = s->d.bc;
  const int L = s->L;
  auto conv_in = [&](long long n) {
    launch_add_conv<double, T>(vref<double>(x), nullptr, vref<T>(s->t), n, nrhs,
                               nullptr, st);
  };
  auto conv_out = [&](long long n) {
    launch_add_conv<T, double>(vref<T>(s->yv), nullptr, vref<double>(y), n, nrhs,
                               nullptr, st);
  };
  C<T>* tin = (C<T>*)s->t;
  C<T>* yout = (C<T>*)s->yv;
  switch (op) {
    case HZ_OP_HELMHOLTZ:
      if (level != 0) break;
      launch_helm<double>(dev64(s, 0), bc, helm1(), vref<double>(x),
                          vref<double>(nullptr), y, nrhs, nullptr, st);
      return cuda_check(s, "apply helmholtz");
    case HZ_OP_CSLP:
      if (level < 0 || level > L) break;
      conv_in(s->lv[level].n);
      launch_helm<T>(s->lv[level].dev(), bc, cslp(s), vref<T>(tin), vref<T>(nullptr),
                     yout, nrhs, nullptr, st);
      conv_out(s->lv[level].n);
      return cuda_check(s, "apply cslp");
    case HZ_OP_VCYCLE:
      if (level < 0 || level > L) break;
      conv_in(s->lv[level].n);
      vcycle<T>(s, level, vref<T>(tin), yout, nrhs, nullptr);
      conv_out(s->lv[level].n);
      return cuda_check(s, "apply vcycle");
    case HZ_OP_RESTRICT_FW:
      if (level < 0 || level >= L) break;
      conv_in(s->lv[level].n);
      launch_restrict_z<T>(s->lv[level].dev(), s->lv[level + 1].dev(), bc, ZK_BILINEAR,
                           vref<T>(tin), yout, nrhs, nullptr, st);
      conv_out(s->lv[level + 1].n);
      return cuda_check(s, "apply restrict");
    case HZ_OP_PROLONG_BILINEAR:
      if (level < 0 || level >= L) break;
      conv_in(s->lv[level + 1].n);
      launch_prolong_z<T>(s->lv[level].dev(), s->lv[level + 1].dev(), bc, ZK_BILINEAR,
                          tin, yout, 0, nrhs, nullptr, st);
      conv_out(s->lv[level].n);
      return cuda_check(s, "apply prolong");
    default:
      break;
  }
  if (s->d.zkind == HZ_Z_NONE) {
    if (op == HZ_OP_PRECOND) {
      hz_status e = precond<T>(s, vref<double>(x), vref<double>(y), nrhs, nullptr);
      return e;
    }
    set_err(s, "operator %d needs deflation vectors (zkind != HZ_Z_NONE) or a "
               "valid level", (int)op);
    return HZ_INVALID_ARG;
  }
  switch (op) {
    case HZ_OP_RESTRICT_Z:
      conv_in(s->lv[0].n);
      launch_restrict_z<T>(s->lv[0].dev(), s->lv[1].dev(), bc, s->d.zkind, vref<T>(tin),
                           yout, nrhs, nullptr, st, rz_scale(s));
      conv_out(s->lv[1].n);
      return cuda_check(s, "apply restrict_z");
    case HZ_OP_PROLONG_Z:
      conv_in(s->lv[1].n);
      launch_prolong_z<T>(s->lv[0].dev(), s->lv[1].dev(), bc, s->d.zkind, tin, yout, 0,
                          nrhs, nullptr, st);
      conv_out(s->lv[0].n);
      return cuda_check(s, "apply prolong_z");
    case HZ_OP_COARSE_E:
      conv_in(s->lv[1].n);
      apply_E<T>(s, tin, yout, nrhs, nullptr);
      conv_out(s->lv[1].n);
      return cuda_check(s, "apply E");
    case HZ_OP_COARSE_SOLVE: {
      conv_in(s->lv[1].n);
      launch_mask_dirichlet<T>(s->lv[1].dev(), bc, tin, nrhs, st);
      hz_status e = coarse_solve<T>(s, tin, yout, nrhs, nullptr);
      if (e != HZ_OK) return e;
      conv_out(s->lv[1].n);
      e = cuda_check(s, "apply coarse solve");
      return e == HZ_OK ? take_fault(s) : e;
    }
    case HZ_OP_PRECOND: {
      const hz_status e = precond<T>(s, vref<double>(x), vref<double>(y), nrhs, nullptr);
      return e == HZ_OK ? take_fault(s) : e;
    }
    default:
      break;
  }
  set_err(s, "invalid operator %d / level %d", (int)op, level);
  return HZ_INVALID_ARG;
}

}  // namespace

// ================================================================= C ABI
extern "C" {

void hz_desc_default(hz_desc* d, int nx, int ny, double h) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->nx = nx;
  d->ny = ny;
  d->h = h;
  d->bc = HZ_BC_SOMMERFELD;
  d->zkind = HZ_Z_HO;
  d->ekind = HZ_E_GALERKIN;
  d->prec = HZ_PREC_FP64;
  d->beta1 = 1.0;
  d->beta2 = -0.5;
  d->jacobi_omega = 0.8;
  d->min_coarse_intervals = 2;
  d->coarse_tol = 1e-6;
  d->coarse_maxit = 500;
  d->outer_maxit = 100;
  d->nrhs_max = 1;
}

hz_status hz_workspace_bytes(const hz_desc* d, size_t* bytes) {
  std::string why;
  if (!bytes || !valid_desc(d, &why)) return HZ_INVALID_ARG;
  hz_solver tmp;
  tmp.d = *d;
  const hz_status e = init_shapes(&tmp);
  if (e != HZ_OK) return e;
  Arena a;
  plan(&tmp, a);
  *bytes = a.off + 256;
  return HZ_OK;
}

hz_status hz_setup(const hz_desc* d, const double* k2_dev, void* ws, size_t ws_bytes,
                   void* stream, hz_solver** out) {
  std::string why;
  if (!out) return HZ_INVALID_ARG;
  *out = nullptr;
  if (!valid_desc(d, &why) || !k2_dev || !ws) return HZ_INVALID_ARG;
  if (((uintptr_t)ws) & 255) return HZ_INVALID_ARG;
  hz_solver* s = new hz_solver();
  s->d = *d;
  hz_tuning_default(&s->tune);
  s->st = (cudaStream_t)stream;
  if (const char* ce = std::getenv("HZ_CHECK_EVERY")) {
    const int v = std::atoi(ce);
    if (v > 0) s->check_every = v;
  }
  hz_status e = init_shapes(s);
  if (e != HZ_OK) {
    delete s;
    return e;
  }
  Arena dry;
  plan(s, dry);
  if (dry.off + 256 > ws_bytes) {
    delete s;
    return HZ_WORKSPACE_TOO_SMALL;
  }
  Arena a;
  a.dry = false;
  a.base = (char*)ws;
  plan(s, a);
  s->ws_bytes = ws_bytes;
  cudaStream_t st = s->st;
  cudaMemcpyAsync(s->lv[0].k2d, k2_dev, sizeof(double) * s->lv[0].n,
                  cudaMemcpyDeviceToDevice, st);
  for (int l = 1; l <= s->L; ++l)
    launch_inject(dev64(s, l - 1), dev64(s, l), s->lv[l].k2d, st);
  const Shift sh = cslp(s);
  for (int l = 0; l <= s->L; ++l) {
    if (s->mixed) launch_cast_k2(s->lv[l].k2d, s->lv[l].k2f, s->lv[l].n, st);
    launch_dinv(dev64(s, l), s->d.bc, sh, s->d.jacobi_omega, s->lv[l].dinv_d,
                s->lv[l].dinv_f, st);
  }
  cudaMemsetAsync(s->gj_err, 0, sizeof(int), st);
  cudaMemsetAsync(s->fault, 0, sizeof(int), st);
  cudaMemsetAsync(s->izero, 0, sizeof(int), st);
  if (s->Sglk) extract_galerkin_stencil(s);
  launch_dense_assemble(dev64(s, s->L), s->d.bc, sh, s->aug, st);
  launch_gauss_jordan(s->nL, s->aug, s->gj_err, st);
  launch_extract_inverse(dev64(s, s->L), s->d.bc, s->aug,
                         s->mixed ? nullptr : (double2*)s->minv,
                         s->mixed ? (float2*)s->minv : nullptr, st);
  int gerr = 0;
  e = cuda_check(s, "setup");
  if (e == HZ_OK) e = read_flag(s, s->gj_err, &gerr);
  if (e == HZ_OK && gerr) {
    set_err(s, "coarsest-level CSLP matrix is singular");
    e = HZ_INVALID_GRID;
  }
  if (e != HZ_OK) {
    delete s;
    return e;
  }
  *out = s;
  return HZ_OK;
}

hz_status hz_solve(hz_solver* s, const void* b_dev, void* x_dev, int nrhs, double tol,
                   int use_x0, hz_solve_info* info) {
  if (!s || !b_dev || !x_dev || nrhs < 1 || nrhs > s->d.nrhs_max || !(tol > 0))
    return HZ_INVALID_ARG;
  return solve_dev(s, (const double2*)b_dev, (double2*)x_dev, nrhs, tol, use_x0, info);
}

hz_status hz_solve_async(hz_solver* s, const void* b_dev, void* x_dev, int nrhs, double tol,
                         int use_x0, hz_solve_info* info_dev) {
  if (!s || !b_dev || !x_dev || !info_dev || nrhs < 1 || nrhs > s->d.nrhs_max ||
      !(tol > 0))
    return HZ_INVALID_ARG;
  if (s->d.outer_solver != HZ_OUTER_FGMRES || s->d.restart > 0 || s->d.no_cuda_graph ||
      s->prof_kc != HZ_KC_NONE) {
    set_err(s, "hz_solve_async needs FGMRES without restart and with CUDA graphs, and no "
               "kernel profiling");
    return HZ_INVALID_ARG;
  }
  return solve_async(s, (const double2*)b_dev, (double2*)x_dev, nrhs, tol, use_x0,
                     (hz_solve_info*)info_dev);
}

hz_status hz_solve_host(hz_solver* s, const void* b_host, void* x_host, int nrhs,
                        double tol, hz_solve_info* info) {
  if (!s || !b_host || !x_host || nrhs < 1 || nrhs > s->d.nrhs_max || !(tol > 0))
    return HZ_INVALID_ARG;
  const size_t bytes = sizeof(double2) * (size_t)s->lv[0].n * nrhs;
  if (cudaMemcpyAsync(s->io0, b_host, bytes, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
    return cuda_check(s, "h2d");
  const hz_status e = solve_dev(s, s->io0, s->io1, nrhs, tol, 0, info);
  if (e != HZ_OK && e != HZ_NOT_CONVERGED && e != HZ_BREAKDOWN) return e;
  if (cudaMemcpyAsync(x_host, s->io1, bytes, cudaMemcpyDeviceToHost, s->st) != cudaSuccess)
    return cuda_check(s, "d2h");
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return cuda_check(s, "d2h sync");
  return e;
}

hz_status hz_apply(hz_solver* s, hz_op op, int level, const void* x_dev, void* y_dev,
                   int nrhs) {
  if (!s || !x_dev || !y_dev || nrhs < 1 || nrhs > s->d.nrhs_max) return HZ_INVALID_ARG;
  return s->mixed ? apply_op<float>(s, op, level, (const double2*)x_dev,
                                    (double2*)y_dev, nrhs)
                  : apply_op<double>(s, op, level, (const double2*)x_dev,
                                     (double2*)y_dev, nrhs);
}

hz_status hz_last_inner_iters(hz_solver* s, int* iters_host, int nrhs) {
  if (!s || !iters_host || nrhs < 1 || nrhs > s->d.nrhs_max) return HZ_INVALID_ARG;
  if (s->d.zkind == HZ_Z_NONE) {
    for (int r = 0; r < nrhs; ++r) iters_host[r] = 0;
    return HZ_OK;
  }
  cudaMemcpyAsync(iters_host, s->kin.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost,
                  s->st);
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return cuda_check(s, "iters");
  return HZ_OK;
}

int hz_num_levels(const hz_solver* s) { return s ? s->L + 1 : 0; }

hz_status hz_level_shape(const hz_solver* s, int level, int* nx, int* ny) {
  if (!s || level < 0 || level > s->L || !nx || !ny) return HZ_INVALID_ARG;
  *nx = s->lv[level].nx;
  *ny = s->lv[level].ny;
  return HZ_OK;
}

hz_status hz_gradient(hz_solver* s, double omega, const void* src_dev, int nshots,
                      const int* rec_idx_dev, int nrec, const void* d_obs_dev,
                      double tol, double* J_host, double* grad_dev,
                      hz_solve_info* info) {
  if (!s || !src_dev || nshots < 1 || !rec_idx_dev || nrec < 1 || !d_obs_dev ||
      !J_host || !grad_dev || !(tol > 0) || !(omega > 0))
    return HZ_INVALID_ARG;
  cudaStream_t st = s->st;
  const long long n0 = s->lv[0].n;
  const int B = s->d.nrhs_max;
  const int bc = s->d.bc;
  cudaMemsetAsync(grad_dev, 0, sizeof(double) * n0, st);
  cudaMemsetAsync(s->Jd, 0, sizeof(double), st);
  hz_status worst = HZ_OK;
  std::vector<hz_solve_info> inf(B);
  for (int s0 = 0; s0 < nshots; s0 += B) {
    const int nb = (nshots - s0 < B) ? nshots - s0 : B;
    const double2* src = (const double2*)src_dev + (long long)s0 * n0;
    hz_status e = solve_dev(s, src, s->io2, nb, tol, 0, inf.data());
    if (e != HZ_OK && e != HZ_NOT_CONVERGED && e != HZ_BREAKDOWN) return e;
    if (worst == HZ_OK) worst = e;
    if (info)
      for (int r = 0; r < nb; ++r) info[2 * (s0 + r)] = inf[r];
    cudaMemsetAsync(s->io0, 0, sizeof(double2) * n0 * nb, st);
    launch_adjoint_source(s->lv[0].nx, s->lv[0].ny, bc, s->io2, rec_idx_dev, nrec,
                          (const double2*)d_obs_dev + (long long)s0 * nrec, s->io0,
                          s->Jd, nb, st);
    e = solve_dev(s, s->io0, s->io1, nb, tol, 0, inf.data());
    if (e != HZ_OK && e != HZ_NOT_CONVERGED && e != HZ_BREAKDOWN) return e;
    if (worst == HZ_OK) worst = e;
    if (info)
      for (int r = 0; r < nb; ++r) info[2 * (s0 + r) + 1] = inf[r];
    launch_image(dev64(s, 0), bc, omega, s->io2, s->io1, grad_dev, nb, st);
  }
  cudaMemcpyAsync(J_host, s->Jd, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(s, "gradient");
  const hz_status e = cuda_check(s, "gradient");
  return e != HZ_OK ? e : worst;
}

hz_status hz_solve_group(hz_solver* const* members, int count, const void* const* b_dev,
                         void* const* x_dev, const int* nrhs, double tol,
                         hz_solve_info* const* info) {
  GroupScope G(members, count);
  if (G.status != HZ_OK) return G.status;
  if (!b_dev || !x_dev || !nrhs || !(tol > 0)) return HZ_INVALID_ARG;
  std::vector<Member> M;
  std::vector<const double2*> b;
  std::vector<double2*> x;
  for (int g = 0; g < count; ++g) {
    if (!b_dev[g] || !x_dev[g] || nrhs[g] < 1 || nrhs[g] > G.S[g]->d.nrhs_max)
      return HZ_INVALID_ARG;
    M.push_back({G.S[g], nrhs[g]});
    b.push_back((const double2*)b_dev[g]);
    x.push_back((double2*)x_dev[g]);
  }
  return solve_group_dev(M, b.data(), x.data(), tol, info, G.S[0]->st);
}

hz_status hz_gradient_group(hz_solver* const* members, int count, const double* omega,
                            const void* const* src_dev, const int* nshots,
                            const int* const* rec_idx_dev, const int* nrec,
                            const void* const* d_obs_dev, double tol, double* J_host,
                            double* const* grad_dev, hz_solve_info* const* info) {
  GroupScope G(members, count);
  if (G.status != HZ_OK) return G.status;
  if (!omega || !src_dev || !nshots || !rec_idx_dev || !nrec || !d_obs_dev || !J_host ||
      !grad_dev || !(tol > 0))
    return HZ_INVALID_ARG;
  for (int g = 0; g < count; ++g)
    if (!(omega[g] > 0) || !src_dev[g] || nshots[g] < 1 || !rec_idx_dev[g] || nrec[g] < 1 ||
        !d_obs_dev[g] || !grad_dev[g])
      return HZ_INVALID_ARG;
  cudaStream_t st = G.S[0]->st;
  for (int g = 0; g < count; ++g) {
    cudaMemsetAsync(grad_dev[g], 0, sizeof(double) * G.S[g]->lv[0].n, st);
    cudaMemsetAsync(G.S[g]->Jd, 0, sizeof(double), st);
  }
  hz_status worst = HZ_OK;
  std::vector<std::vector<hz_solve_info>> inf(count);
  for (int k = 0;; ++k) {
    // batch k: shots k*B .. of every member that has any left
    std::vector<Member> M;
    std::vector<int> gi, s0;
    std::vector<const double2*> b;
    std::vector<double2*> x;
    std::vector<hz_solve_info*> ip;
    for (int g = 0; g < count; ++g) {
      hz_solver* s = G.S[g];
      const int B = s->d.nrhs_max, first = k * B;
      if (first >= nshots[g]) continue;
      const int nb = nshots[g] - first < B ? nshots[g] - first : B;
      M.push_back({s, nb});
      gi.push_back(g);
      s0.push_back(first);
      inf[g].resize(B);
    }
    if (M.empty()) break;
    for (size_t a = 0; a < M.size(); ++a) {
      hz_solver* s = M[a].s;
      b.push_back((const double2*)src_dev[gi[a]] + (long long)s0[a] * s->lv[0].n);
      x.push_back(s->io2);
      ip.push_back(inf[gi[a]].data());
    }
    hz_status e = solve_group_dev(M, b.data(), x.data(), tol, ip.data(), st);
    if (e != HZ_OK && e != HZ_NOT_CONVERGED && e != HZ_BREAKDOWN) return e;
    if (worst == HZ_OK) worst = e;
    for (size_t a = 0; a < M.size(); ++a) {
      hz_solver* s = M[a].s;
      const int g = gi[a];
      if (info && info[g])
        for (int r = 0; r < M[a].nrhs; ++r) info[g][2 * (s0[a] + r)] = inf[g][r];
      const long long n0 = s->lv[0].n;
      cudaMemsetAsync(s->io0, 0, sizeof(double2) * n0 * M[a].nrhs, st);
      launch_adjoint_source(s->lv[0].nx, s->lv[0].ny, s->d.bc, s->io2, rec_idx_dev[g],
                            nrec[g], (const double2*)d_obs_dev[g] + (long long)s0[a] * nrec[g],
                            s->io0, s->Jd, M[a].nrhs, st);
      b[a] = s->io0;
      x[a] = s->io1;
    }
    e = solve_group_dev(M, b.data(), x.data(), tol, ip.data(), st);
    if (e != HZ_OK && e != HZ_NOT_CONVERGED && e != HZ_BREAKDOWN) return e;
    if (worst == HZ_OK) worst = e;
    for (size_t a = 0; a < M.size(); ++a) {
      hz_solver* s = M[a].s;
      const int g = gi[a];
      if (info && info[g])
        for (int r = 0; r < M[a].nrhs; ++r) info[g][2 * (s0[a] + r) + 1] = inf[g][r];
      launch_image(dev64(s, 0), s->d.bc, omega[g], s->io2, s->io1, grad_dev[g], M[a].nrhs,
                   st);
    }
  }
  for (int g = 0; g < count; ++g)
    cudaMemcpyAsync(&J_host[g], G.S[g]->Jd, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(G.S[0], "gradient group");
  const hz_status e = cuda_check(G.S[0], "gradient group");
  return e != HZ_OK ? e : worst;
}

hz_status hz_profile_begin(hz_solver* s, hz_kernel_class kc, int max_launches) {
  if (!s || kc < HZ_KC_NONE || kc > HZ_KC_VCYCLE || max_launches < 0)
    return HZ_INVALID_ARG;
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  s->prof_ev.clear();
  s->prof_used = 0;
  s->prof_dropped = 0;
  s->prof_kc = HZ_KC_NONE;
  if (kc == HZ_KC_NONE) return HZ_OK;
  s->prof_ev.resize(2 * (size_t)max_launches);
  for (auto& e : s->prof_ev)
    if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(s, "profile events");
  cudaMemsetAsync(s->prof_bytes, 0, sizeof(unsigned long long), s->st);
  s->prof_kc = kc;
  return cuda_check(s, "profile begin");
}

hz_status hz_profile_end(hz_solver* s, long long* launches, double* ms_total,
                         double* alg_bytes) {
  if (!s || !launches || !ms_total || !alg_bytes) return HZ_INVALID_ARG;
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return cuda_check(s, "profile sync");
  double ms = 0.0;
  const size_t pairs = s->prof_used / 2;
  for (size_t p = 0; p < pairs; ++p) {
    float t = 0.f;
    cudaEventElapsedTime(&t, s->prof_ev[2 * p], s->prof_ev[2 * p + 1]);
    ms += t;
  }
  unsigned long long b = 0;
  cudaMemcpy(&b, s->prof_bytes, sizeof(b), cudaMemcpyDeviceToHost);
  *launches = (long long)pairs;
  *ms_total = ms;
  *alg_bytes = (double)b;
  const bool complete = s->prof_dropped == 0;
  hz_profile_begin(s, HZ_KC_NONE, 0);
  if (!complete) {
    set_err(s, "profile event pool too small: launches dropped");
    return HZ_INVALID_ARG;
  }
  return cuda_check(s, "profile end");
}

hz_status hz_destroy(hz_solver* s) {
  if (s) hz_profile_begin(s, HZ_KC_NONE, 0);
  delete s;
  return HZ_OK;
}

const char* hz_status_str(hz_status st) {
  switch (st) {
    case HZ_OK: return "ok";
    case HZ_INVALID_ARG: return "invalid argument";
    case HZ_INVALID_GRID: return "invalid grid";
    case HZ_WORKSPACE_TOO_SMALL: return "workspace too small";
    case HZ_NOT_CONVERGED: return "not converged";
    case HZ_BREAKDOWN: return "breakdown";
    case HZ_NAN: return "NaN or Inf in a residual";
    case HZ_TIMEOUT: return "timeout";
    case HZ_CUDA_ERROR: return "CUDA error";
  }
  return "unknown status";
}

const char* hz_last_error(const hz_solver* s) { return s ? s->err.c_str() : ""; }

void hz_tuning_default(hz_tuning* t) {
  if (!t) return;
  std::memset(t, 0, sizeof(*t));
  t->mdot_kernel = 0;
  t->maxpy_kernel = 0;
  t->galerkin_apply = 0;
  t->e_rhs_per_block = 0;
  t->vcycle_fused = 0;
  t->vcycle_rhs_per_block = 0;
  t->vcycle_tile = 0;
  t->e_column_pairs = 0;
}

hz_status hz_get_tuning(const hz_solver* s, hz_tuning* t) {
  if (!s || !t) return HZ_INVALID_ARG;
  *t = s->tune;
  return HZ_OK;
}

hz_status hz_set_tuning(hz_solver* s, const hz_tuning* t) {
  if (!s || !t || t->mdot_kernel < 0 || t->mdot_kernel > 2 || t->maxpy_kernel < 0 ||
      t->maxpy_kernel > 2 || t->galerkin_apply < 0 || t->galerkin_apply > 1 ||
      t->e_rhs_per_block < 0 || t->e_rhs_per_block > kMaxRhs || t->vcycle_fused < 0 ||
      t->vcycle_fused > 2 || t->vcycle_rhs_per_block < 0 ||
      t->vcycle_rhs_per_block > kMaxRhs || t->vcycle_tile < 0 || t->vcycle_tile > 1 ||
      t->e_column_pairs < 0 || t->e_column_pairs > 1)
    return HZ_INVALID_ARG;
  if (t->galerkin_apply == 1 && !s->Sglk) {
    set_err(s, "galerkin_apply = 1 needs the Galerkin coarse operator (HZ_E_GALERKIN)");
    return HZ_INVALID_ARG;
  }
  // captured graphs hold the launches of the previous choice
  if (!s->graphs.empty()) {
    cudaStreamSynchronize(s->st);
    for (hz_solver::OuterGraph& g : s->graphs) {
      cudaGraphExecDestroy(g.ex);
      cudaGraphDestroy(g.g);
    }
    s->graphs.clear();
  }
  s->tune = *t;
  s->kin.dotk = s->kout.dotk = t->mdot_kernel;
  s->kin.updk = s->kout.updk = t->maxpy_kernel;
  for (int l = 2; l <= s->D; ++l) {
    s->dl[l].ks.dotk = t->mdot_kernel;
    s->dl[l].ks.updk = t->maxpy_kernel;
  }
  return HZ_OK;
}

// staged V-cycle candidates: RHS per block x prolongation tile
constexpr int kVcycleRpb[3] = {4, 8, 16};
constexpr int kVcycleStaged = 6;
static_assert(11 + 2 + kVcycleStaged + 1 == HZ_TUNE_CANDIDATES, "candidate count");

hz_status hz_autotune(hz_solver* s, int nrhs, hz_tuning* best, double* ms) {
  if (!s || nrhs < 1 || nrhs > s->d.nrhs_max) return HZ_INVALID_ARG;
  const int saved_prof = s->prof_kc;
  s->prof_kc = HZ_KC_NONE;
  hz_tuning t = s->tune;
  double tm[HZ_TUNE_CANDIDATES];
  for (double& v : tm) v = -1.0;
  for (int upd = 0; upd <= 1; ++upd) {
    int pick = 0;
    for (int v = 0; v <= 2; ++v) {
      tm[3 * upd + v] = time_cgs_any(s, nrhs, upd != 0, v);
      if (tm[3 * upd + v] < tm[3 * upd + pick]) pick = v;
    }
    (upd ? t.maxpy_kernel : t.mdot_kernel) = pick;
  }
  if (s->Sglk) {
    const int rpb[3] = {0, 8, 4};
    int pick = 0;
    for (int k = 0; k < 3; ++k) {
      tm[8 + k] = s->mixed ? time_e<float>(s, nrhs, 1, rpb[k], 0)
                           : time_e<double>(s, nrhs, 1, rpb[k], 0);
      if (tm[8 + k] < tm[8 + pick]) pick = k;
    }
    t.e_rhs_per_block = rpb[pick];
    tm[19] = s->mixed ? time_e<float>(s, nrhs, 1, rpb[pick], 1)
                      : time_e<double>(s, nrhs, 1, rpb[pick], 1);
    t.e_column_pairs = tm[19] < tm[8 + pick] ? 1 : 0;
    tm[6] = s->mixed ? time_e<float>(s, nrhs, 0, 0, 0) : time_e<double>(s, nrhs, 0, 0, 0);
    tm[7] = t.e_column_pairs ? tm[19] : tm[8 + pick];
    t.galerkin_apply = tm[7] < tm[6] ? 1 : 0;
  }
  if (s->L >= 1) {
    // separate, fused, then the staged multi-RHS kernels for each
    // (RHS per block, prolongation tile) of kVcycleStaged
    int pick = 0;
    for (int c = 0; c < 2 + kVcycleStaged; ++c) {
      const int f = c < 2 ? c : 2;
      const int rpb = c < 2 ? 0 : kVcycleRpb[(c - 2) % 3];
      const int tile = c < 2 ? 0 : (c - 2) / 3;
      tm[11 + c] = s->mixed ? time_vcycle<float>(s, nrhs, f, rpb, tile)
                            : time_vcycle<double>(s, nrhs, f, rpb, tile);
      if (tm[11 + c] < tm[11 + pick]) pick = c;
    }
    t.vcycle_fused = pick < 2 ? pick : 2;
    if (pick >= 2) {
      t.vcycle_rhs_per_block = kVcycleRpb[(pick - 2) % 3];
      t.vcycle_tile = (pick - 2) / 3;
    }
  }
  s->prof_kc = saved_prof;
  hz_status e = take_fault(s);
  if (e == HZ_OK) e = cuda_check(s, "autotune");
  if (e != HZ_OK) return e;
  e = hz_set_tuning(s, &t);
  if (e != HZ_OK) return e;
  if (best) *best = t;
  if (ms)
    for (int k = 0; k < HZ_TUNE_CANDIDATES; ++k) ms[k] = tm[k];
  return HZ_OK;
}

hz_status hz_fault_drill(hz_solver* s, int starve_copies, double wait_seconds) {
  if (!s || !(wait_seconds > 0) || wait_seconds > 2.0) return HZ_INVALID_ARG;
  const unsigned long long ns = (unsigned long long)(wait_seconds * 1e9);
  auto set = [&](KState& k) {
    k.starve = starve_copies ? 1 : 0;
    k.wait_ns = ns;
  };
  set(s->kin);
  set(s->kout);
  for (int l = 2; l <= s->D; ++l) set(s->dl[l].ks);
  // captured graphs hold the previous kernel arguments
  if (!s->graphs.empty()) {
    cudaStreamSynchronize(s->st);
    for (hz_solver::OuterGraph& g : s->graphs) {
      cudaGraphExecDestroy(g.ex);
      cudaGraphDestroy(g.g);
    }
    s->graphs.clear();
  }
  return HZ_OK;
}

long long hz_host_launches(void) { return hz::host_op_counter().load(); }

long long hz_kernel_launches(void) {
  long long n = hz::launch_counter().load();
  if (g_graph_launched.load()) n += (long long)hz::graph_body_kernels_run();
  return n;
}

}  // extern "C"
