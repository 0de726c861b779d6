// Internal types and device helpers shared by the CUDA translation units of
// libhz.so.  Complex numbers are double2 / float2 (x = real, y = imag).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace hz {

// Number of kernels this library has launched (all launchers count), and
// of launch operations the host issued (a kernel launched directly or a
// CUDA graph launched counts one each).
inline std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}
inline std::atomic<long long>& host_op_counter() {
  static std::atomic<long long> c{0};
  return c;
}
#define HZ_COUNT()                                                       \
  (::hz::launch_counter().fetch_add(1, std::memory_order_relaxed),      \
   ::hz::host_op_counter().fetch_add(1, std::memory_order_relaxed))

enum { BC_DIRICHLET = 0, BC_SOMMERFELD = 1 };
enum { ZK_NONE = 0, ZK_BILINEAR = 1, ZK_HO = 2 };
enum { EK_GALERKIN = 0, EK_RED_O2 = 1, EK_RED_GLK1 = 2, EK_RED_GLK2 = 3 };

template <class T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };
template <class T> using C = typename CT<T>::t;

__host__ __device__ __forceinline__ double2 mkc(double r, double i) {
  return make_double2(r, i);
}
__host__ __device__ __forceinline__ float2 mkc(float r, float i) {
  return make_float2(r, i);
}
template <class T> __host__ __device__ __forceinline__ C<T> czero() {
  return mkc(T(0), T(0));
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 operator-(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 operator*(double s, double2 a) {
  return make_double2(s * a.x, s * a.y);
}
__device__ __forceinline__ float2 operator*(float s, float2 a) {
  return make_float2(s * a.x, s * a.y);
}
// complex product
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)),
                      fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)),
                     fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
// acc + s * a (s real)
__device__ __forceinline__ double2 rfma(double s, double2 a, double2 acc) {
  return make_double2(fma(s, a.x, acc.x), fma(s, a.y, acc.y));
}
__device__ __forceinline__ float2 rfma(float s, float2 a, float2 acc) {
  return make_float2(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y));
}

// Level descriptor passed by value to kernels.
struct LevelDev {
  int nx, ny;
  double h;
  double ih2d, tihd;      // 1/h^2 and 2/h
  float ih2f, tihf;
  const double* k2d;      // k^2, FP64
  const float* k2f;       // k^2, FP32 (mixed precision only)
  const double2* dinv_d;  // omega / diag(M), FP64 precision path
  const float2* dinv_f;   // omega / diag(M), FP32 precision path
};

template <class T> __device__ __forceinline__ const T* k2_of(const LevelDev& L);
template <> __device__ __forceinline__ const double* k2_of<double>(const LevelDev& L) {
  return L.k2d;
}
template <> __device__ __forceinline__ const float* k2_of<float>(const LevelDev& L) {
  return L.k2f;
}
template <class T> __device__ __forceinline__ T ih2_of(const LevelDev& L);
template <> __device__ __forceinline__ double ih2_of<double>(const LevelDev& L) {
  return L.ih2d;
}
template <> __device__ __forceinline__ float ih2_of<float>(const LevelDev& L) {
  return L.ih2f;
}
template <class T> __device__ __forceinline__ T tih_of(const LevelDev& L);
template <> __device__ __forceinline__ double tih_of<double>(const LevelDev& L) {
  return L.tihd;
}
template <> __device__ __forceinline__ float tih_of<float>(const LevelDev& L) {
  return L.tihf;
}
template <class T> __device__ __forceinline__ const C<T>* dinv_of(const LevelDev& L);
template <> __device__ __forceinline__ const double2* dinv_of<double>(const LevelDev& L) {
  return L.dinv_d;
}
template <> __device__ __forceinline__ const float2* dinv_of<float>(const LevelDev& L) {
  return L.dinv_f;
}

// A vector argument whose base may be indexed by a device-side counter:
// the vector used is base + (*jidx + jofs) * jstride (jidx may be null).
// Lets one launch configuration serve every iteration of a Krylov loop.
// E is the stored element type (double2, float2 or __half2).
template <class E> struct VRefE {
  E* base;
  const int* jidx;
  int jofs;
  long long jstride;
  __device__ __forceinline__ E* get() const {
    return jidx ? base + (long long)(*jidx + jofs) * jstride : base;
  }
};
template <class T> using VRef = VRefE<C<T>>;
template <class E> inline VRefE<E> vrefe(const void* p) {
  VRefE<E> r;
  r.base = (E*)p;
  r.jidx = nullptr;
  r.jofs = 0;
  r.jstride = 0;
  return r;
}
template <class E>
inline VRefE<E> vrefe_j(const void* p, const int* jidx, int jofs, long long stride) {
  VRefE<E> r;
  r.base = (E*)p;
  r.jidx = jidx;
  r.jofs = jofs;
  r.jstride = stride;
  return r;
}
template <class T> inline VRef<T> vref(const void* p) { return vrefe<C<T>>(p); }
template <class T>
inline VRef<T> vref_j(const void* p, const int* jidx, int jofs, long long stride) {
  return vrefe_j<C<T>>(p, jidx, jofs, stride);
}

// Loads and stores of a complex value kept in storage type E, computed in
// the matching double2 / float2 (an FP16 pair is computed in FP32).
__device__ __forceinline__ double2 ld2(const double2* p, long long i) { return p[i]; }
__device__ __forceinline__ float2 ld2(const float2* p, long long i) { return p[i]; }
__device__ __forceinline__ float2 ld2(const __half2* p, long long i) {
  return __half22float2(p[i]);
}
__device__ __forceinline__ void st2(double2* p, long long i, double2 v) { p[i] = v; }
__device__ __forceinline__ void st2(float2* p, long long i, float2 v) { p[i] = v; }
__device__ __forceinline__ void st2(__half2* p, long long i, float2 v) {
  p[i] = __float22half2_rn(v);
}

// ---------------------------------------------------------------------
// launchers (defined in hz_stencil.cu / hz_krylov.cu, instantiated for
// float and double)
// ---------------------------------------------------------------------
struct Shift {
  double re, im;
};

// y = op(x) or y = b - op(x), op = -Lap_h - shift k^2 (+ Sommerfeld rows)
template <class T>
void launch_helm(const LevelDev& L, int bc, Shift s, VRef<T> x, VRef<T> b,
                 C<T>* y, int nrhs, const int* done, cudaStream_t st);
// V-cycle kernels (hz_vcycle.cu).  SF: storage of the level right-hand side
// f, SX: storage of the level iterate, SC: storage of the coarse vector,
// SO: storage of the output; the arithmetic is C<T>.
// x = dinv .* f
template <class T, class SF, class SX>
void launch_jacobi0(const LevelDev& L, int bc, VRefE<SF> f, SX* x, int nrhs,
                    const int* done, cudaStream_t st);
// fc = R_fw (f - M x)
template <class T, class SF, class SX, class SC>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc,
                           Shift s, VRefE<SF> f, const SX* x, SC* fc, int nrhs,
                           const int* done, cudaStream_t st);
// x += P_bilinear xc
template <class T, class SC, class SX>
void launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, int bc,
                        const SC* xc, SX* x, int nrhs, const int* done,
                        cudaStream_t st);
// xo = x + dinv .* (f - M x)
template <class T, class SF, class SX, class SO>
void launch_smooth(const LevelDev& L, int bc, Shift s, VRefE<SF> f, const SX* x,
                   SO* xo, int nrhs, const int* done, cudaStream_t st);
// fused: x = dinv .* f and fc = R_FW (f - M x) in one pass over a tile
template <class T, class SF, class SX, class SC>
void launch_pre_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                         VRefE<SF> f, SX* x, SC* fc, int nrhs, const int* done,
                         cudaStream_t st);
// fused: xo = x' + dinv .* (f - M x') with x' = x + P xc
template <class T, class SC, class SX, class SF, class SO>
void launch_prolong_smooth(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                           const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                           const int* done, cudaStream_t st);
// the same two fused kernels, each block walking over a group of rpb
// right-hand sides (0 = all) with its per-node constants in registers and
// the input tiles staged ahead in shared memory (cp.async ring); omega is
// the Jacobi weight D^-1 was built with (the kernels use D^-1 diag(M) =
// omega); prolongation tile 0 = 32 x 8 fine nodes, 1 = 64 x 8
// (abytes, if not null, accumulates the algorithmic bytes of the launch;
// frs is the distance between the right-hand sides of f, 0 = nx * ny)
template <class T, class SF, class SX, class SC>
void launch_pre_restrict_mr(const LevelDev& Lf, const LevelDev& Lc, int bc, double omega,
                            VRefE<SF> f, SX* x, SC* fc, int nrhs, int rpb, const int* done,
                            cudaStream_t st, unsigned long long* abytes = nullptr,
                            long long frs = 0);
template <class T, class SC, class SX, class SF, class SO>
void launch_prolong_smooth_mr(const LevelDev& Lf, const LevelDev& Lc, int bc, double omega,
                              const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                              int rpb, int tile, const int* done, cudaStream_t st,
                              unsigned long long* abytes = nullptr, long long frs = 0);
// x = Minv f on the coarsest level (dense)
// The small levels of a V-cycle in one kernel (complex-FP32 preconditioner):
// levels lv[0..nlev-1] of the hierarchy's tail, the last the coarsest (nL
// nodes, dense inverse); off[k] is level k's first value in shared memory
// (its f, x and a scratch vector follow each other).
constexpr int kMaxSmallLevels = 12;
constexpr int kSmallLevelBytes = 96 * 1024;
struct SmallLevels {
  int nlev, bc, nL;
  float omc;
  LevelDev lv[kMaxSmallLevels];
  int off[kMaxSmallLevels];
  int bytes;
};
template <class SL>
void launch_vcycle_small(const SmallLevels& d, const SL* f, SL* x, const float2* minv,
                         int nrhs, const int* done, cudaStream_t st);

template <class T, class SF, class SO>
void launch_dense_mv(int n, const C<T>* minv, VRefE<SF> f, SO* x, int nrhs,
                     const int* done, cudaStream_t st);
// coarse = scale * R_Z fine  (zk = bilinear: full weighting; ho: 5x5 / 256;
// scale 4 gives the unscaled Z^T)
template <class T>
void launch_restrict_z(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                       VRef<T> fine, C<T>* coarse, int nrhs, const int* done,
                       cudaStream_t st, double scale = 1.0);
// fine = Z coarse (or fine += Z coarse when add != 0)
template <class T>
void launch_prolong_z(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                      const C<T>* coarse, C<T>* fine, int add, int nrhs,
                      const int* done, cudaStream_t st);
// y = R_Z A_h Z x (str-Glk) in one fused tiled kernel
template <class T>
void launch_galerkin_fused(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                           const C<T>* x, C<T>* y, int nrhs, const int* done,
                           cudaStream_t st);
// stcl-op-Glk: probes (FP64) for extracting the Galerkin stencil, the
// extraction into (2R+1)^2 coefficient planes S, and y = E x with them
void launch_probe_fill(const LevelDev& Lc, int P, int c0, int nprobe, double2* out,
                       cudaStream_t st);
template <class T>
void launch_probe_extract(const LevelDev& Lc, int P, int c0, int nprobe,
                          const double2* ep, C<T>* S, cudaStream_t st);
// (pairs: two nodes of a column per thread; rpb: right-hand sides per
// block, 0 = all)
template <class T>
void launch_stencil_e(const LevelDev& Lc, int R, int pairs, const C<T>* S, const C<T>* x,
                      C<T>* y, int nrhs, int rpb, const int* done, cudaStream_t st);
// y = E x with ReD-O4 (4th-order cross, O2 near the boundary) or ReD-cmpO4
// (compact 4th-order 3x3 with 4th-order Sommerfeld ghosts)
template <class T>
void launch_red_o4(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                   const int* done, cudaStream_t st);
template <class T>
void launch_red_cmpo4(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                      const int* done, cudaStream_t st);
// ReD-O6 (sixth-order cross) and ReD-9ptO2 (Appendix B compact scheme)
template <class T>
void launch_red_o6(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                   const int* done, cudaStream_t st);
template <class T>
void launch_red_9pt(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                    const int* done, cudaStream_t st);
// y = E_glk x on level 1 (variant 1 or 2); the 5x5 rows are multiplied by
// gscale (4: the stencil as printed, on the scale of Z^T A Z), the ReD-O2
// boundary rows are not
template <class T>
void launch_glk(const LevelDev& L, int bc, int variant, const C<T>* x, C<T>* y,
                int nrhs, const int* done, cudaStream_t st, double gscale = 1.0);
// zero the Dirichlet boundary nodes of nrhs vectors in place (no-op for
// Sommerfeld grids)
template <class T>
void launch_mask_dirichlet(const LevelDev& L, int bc, C<T>* x, int nrhs,
                           cudaStream_t st);

// out = a + b (b may be null), with conversion of the precision
template <class Ti, class To>
void launch_add_conv(VRef<Ti> a, const C<Ti>* b, VRef<To> out, long long n,
                     int nrhs, const int* done, cudaStream_t st);
// out = a - b
template <class T>
void launch_sub(const C<T>* a, const C<T>* b, C<T>* out, long long n, int nrhs,
                const int* done, cudaStream_t st);
// out = a - b + c, widened to FP64
template <class T>
void launch_sub_add_widen(const C<T>* a, const C<T>* b, const C<T>* c, VRef<double> out,
                          long long n, int nrhs, const int* done, cudaStream_t st);
// setup helpers
void launch_inject(const LevelDev& Lf, const LevelDev& Lc, double* k2c,
                   cudaStream_t st);
void launch_cast_k2(const double* k2d, float* k2f, long long n, cudaStream_t st);
void launch_dinv(const LevelDev& L, int bc, Shift s, double omega, double2* dd,
                 float2* df, cudaStream_t st);
void launch_dense_assemble(const LevelDev& L, int bc, Shift s, double2* aug,
                           cudaStream_t st);
void launch_gauss_jordan(int n, double2* aug, int* err, cudaStream_t st);
// inverse = right half of [I | M^-1]; rows and columns of Dirichlet
// boundary nodes are zeroed (those nodes are not unknowns)
void launch_extract_inverse(const LevelDev& L, int bc, const double2* aug,
                            double2* md, float2* mf, cudaStream_t st);

// Krylov kernels (basis precision T, scalars FP64)
struct KState {
  // per-RHS arrays of length nrhs_max unless noted
  int* jctr;        // [1] current Arnoldi column
  int* done;        // 1 once the RHS stopped iterating
  int* iters;       // iterations taken
  int* stat;        // hz_status per RHS
  int* alldone;     // [1]
  double* bnorm;    // ||b|| (stopping reference)
  double* beta;     // ||r0||
  double* hnorm;    // ||w|| of the current column
  double2* H;       // [nrhs_max][m+1][m] column j at H[(b*(m+1)+i)*m + j]
  double2* g;       // [nrhs_max][m+1]
  double* cs;       // [nrhs_max][m]
  double2* sn;      // [nrhs_max][m]
  double2* y;       // [nrhs_max][m]
  double2* hcol;    // [nrhs_max][m+1] scratch column (one CGS pass)
  double2* part;    // partial sums [nrhs_max][m+1][nblk_max]
  double* npart;    // partial squared norms [nrhs_max][nblk_max]
  double* wpart;    // partial ||w||^2 before projection [nrhs_max][nblk_max]
  int* reorth;      // second Gram-Schmidt pass needed [nrhs_max]
  unsigned long long* abytes;  // [1] algorithmic-byte counter or null
  int* fault;       // [1] set when a pipeline wait of a Krylov kernel timed out
  int dotk, updk;   // multi-dot / multi-update kernels: 0 register-pipelined,
                    // 1 / 2 TMA ring with 8 / 16 consumer warps
  unsigned long long wait_ns;   // bound of every pipeline wait (2 s)
  int starve;       // fault drill: the TMA producers issue no copies, so
                    // the consumers' bounded waits run out
  int m;            // basis size (max iterations)
  int nblk_max;
};

int krylov_nblk(long long n);
// classical Gram-Schmidt pass `pass` (0, or 1 = re-orthogonalisation for
// the RHS flagged by launch_reorth_decide); the basis V is stored as SB,
// w and the arithmetic are C<T>
template <class T, class SB>
void launch_mdot(const SB* V, long long vstride, long long rs, const C<T>* w,
                 long long n, int nrhs, const KState& ks, int pass, cudaStream_t st);
void launch_reduce_cols(const KState& ks, long long n, int nrhs, int pass,
                        cudaStream_t st);
template <class T, class SB>
void launch_maxpy(const SB* V, long long vstride, long long rs, C<T>* w,
                  long long n, int nrhs, const KState& ks, int pass, cudaStream_t st);
void launch_reorth_decide(const KState& ks, long long n, int nrhs, double eta,
                          cudaStream_t st);
template <class T>
void launch_norm2_part(VRef<T> w, long long n, int nrhs, const KState& ks,
                       const int* done, cudaStream_t st);
void launch_reduce_norm(const KState& ks, long long n, int nrhs, double* out,
                        int sqrt_it, cudaStream_t st);
void launch_krylov_init(const KState& ks, int nrhs, const int* done_in,
                        const double* bnorm_src, double tol, cudaStream_t st);
// out = w / s[r], stored as SB (and, if copy is not null, also as C<T> in
// copy [nrhs][n])
template <class T, class SB>
void launch_scale_into(VRef<T> w, VRefE<SB> out, long long rs, const double* s,
                       long long n, int nrhs, const int* done, cudaStream_t st,
                       C<T>* copy = nullptr);
void launch_givens(const KState& ks, int nrhs, double tol, int maxit,
                   cudaStream_t st);
void launch_trisolve(const KState& ks, int nrhs, cudaStream_t st);
// Basis rows: vector i of RHS r starts at V + i * vstride + r * rs; rs is a
// multiple of 4 elements for 16-byte-aligned group loads (or n for FP64).
template <class SB, class Tx>
void launch_update(const SB* V, long long vstride, long long rs, const KState& ks,
                   C<Tx>* x, int accumulate, long long n, int nrhs,
                   cudaStream_t st);
void launch_fill_int(int* p, int v, int count, cudaStream_t st);
// total[r] += iters[r], maxv[r] = max(maxv[r], iters[r]) for RHS not masked
void launch_accum_iters(const int* iters, int* total, int* maxv, int nrhs,
                        const int* mask, cudaStream_t st);
// gradient: adjoint source conj(D^-1 S^T (S u - d)) and misfit J
void launch_adjoint_source(int nx, int ny, int bc, const double2* u,
                           const int* rec, int nrec, const double2* d,
                           double2* adj, double* J, int nrhs, cudaStream_t st);
// grad[n] += -sum_r Re(D_n x_r[n] dA_nn/dm_n u_r[n])
void launch_image(const LevelDev& L, int bc, double omega, const double2* u,
                  const double2* x, double* grad, int nrhs, cudaStream_t st);
void launch_copy_int(const int* src, int* dst, int count, cudaStream_t st);

// Grids of different sizes in one launch: the Gram-Schmidt kernels of up to
// kMaxGroup solvers (each with its own basis, w, n and Krylov state) run as
// one persistent launch over the concatenation of the members' (RHS, chunk)
// tiles; start[g] is the first global tile of member g.
constexpr int kMaxGroup = 8;   // HZ_MAX_GROUP
struct GroupMember {
  const void* V;        // basis (SB), vector i of RHS r at V + i*vstride + r*rs
  long long vstride, rs;
  void* w;              // C<T> [nrhs][n]
  long long n;
  KState ks;
  int nrhs, nblk;
};
struct GroupDesc {
  int count;
  long long start[kMaxGroup + 1];
  GroupMember m[kMaxGroup];
};
template <class T, class SB>
void launch_mdot_group(const GroupDesc& gd, int pass, cudaStream_t st);
template <class T, class SB>
void launch_maxpy_group(const GroupDesc& gd, int pass, cudaStream_t st);

// Flexible GCR outer iteration: x += g u, r -= g c with g = hcol[r][0] and
// partial ||r||^2 in npart; then the convergence test of step k
void launch_gcr_update(double2* x, double2* r, const double2* u, const double2* c,
                       long long n, int nrhs, const KState& ks, cudaStream_t st);
void launch_gcr_check(const KState& ks, const double* rnorm, int nrhs, double tol, int k,
                      int maxit, cudaStream_t st);

// Timing support for the autotuner: synthetic vector contents and an
// Arnoldi state at column j with RHS 0..nrhs-1 active.
template <class SB>
void launch_tune_fill(SB* p, long long count, unsigned seed, cudaStream_t st);
void launch_tune_state(const KState& ks, int nrhs, int j, cudaStream_t st);

// Device-side loop control of an iteration captured as the body of a CUDA
// graph WHILE node.  loop_begin (upstream of the node) resets the iteration
// counter *it and runs the body only if *alldone is clear; loop_next (last
// node of the body) counts the iteration, adds *body_kernels to the device
// total of graph-executed kernels and repeats while *alldone is clear and
// fewer than maxit iterations ran.
void launch_loop_begin(const int* alldone, const int* fault, int* it,
                       cudaGraphConditionalHandle h, cudaStream_t st);
void launch_loop_next(const int* alldone, const int* fault, int* it, int maxit,
                      const int* body_kernels, cudaGraphConditionalHandle h,
                      cudaStream_t st);
// *out = 1 if every flag of fs is set, else 0 (the all-converged flag of a
// group of solvers)
struct FlagSet {
  const int* f[8];
  int n;
};
void launch_all_of(const FlagSet& fs, int* out, cudaStream_t st);
// Kernels run by WHILE-node bodies on the current device so far (0 if the
// counter cannot be read).
unsigned long long graph_body_kernels_run();

}  // namespace hz
