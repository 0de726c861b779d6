// Kernels of the CSLP multigrid V-cycle (Sec. 3.1, Sec. 5.1): damped-Jacobi
// sweeps (w = 0.8) with the residual fused into full-weighting restriction
// (eq. weight operator), bilinear interpolation of the correction (eq.
// bilinear operator) and the dense coarsest-level solve.  Vectors of the
// level hierarchy may be stored in a narrower type than the arithmetic
// (BF16 pairs for the smoother variant); the arithmetic is C<T>.
#include "hz_common.cuh"
#include "hz_stencil_dev.cuh"

namespace hz {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2d(int nx, int ny, int nrhs) {
  return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nrhs);
}

// x = dinv .* f (one damped-Jacobi sweep from x = 0)
template <class T, class SF, class SX>
__global__ void k_jacobi0(LevelDev L, int bc, VRefE<SF> fin, SX* __restrict__ x,
                          const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    st2(x, r * n + id, czero<T>());
    return;
  }
  st2(x, r * n + id, cmul(dinv_of<T>(L)[id], ld2(fin.get(), r * n + id)));
}

// fc(I,J) = sum_{a,b in -1..1} (2-|a|)(2-|b|)/16 * (f - M x)(2I+a, 2J+b)
template <class T, class SF, class SX, class SC>
__global__ void k_resid_restrict(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim,
                                 VRefE<SF> fin, const SX* __restrict__ x,
                                 SC* __restrict__ fc, const int* __restrict__ done) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny || (done && done[r])) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long idc = (long long)J * Lc.nx + I;
  if (bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny)) {
    st2(fc, r * nc + idc, czero<T>());
    return;
  }
  const SF* f = fin.get() + r * nf;
  const SX* xr = x + r * nf;
  C<T> acc = czero<T>();
  for (int b = -1; b <= 1; ++b) {
    const int jf = 2 * J + b;
    if (jf < 0 || jf >= Lf.ny) continue;
    for (int a = -1; a <= 1; ++a) {
      const int ifn = 2 * I + a;
      if (ifn < 0 || ifn >= Lf.nx) continue;
      if (bc == BC_DIRICHLET && on_bnd(ifn, jf, Lf.nx, Lf.ny)) continue;
      const C<T> res = ld2(f, (long long)jf * Lf.nx + ifn) -
                       helm_point<T, SX>(Lf, bc, sre, sim, xr, ifn, jf);
      const T w = T((2 - abs(a)) * (2 - abs(b))) * T(0.0625);
      acc = rfma(w, res, acc);
    }
  }
  st2(fc, r * nc + idc, acc);
}

// x += P_bilinear xc
template <class T, class SC, class SX>
__global__ void k_prolong_add(LevelDev Lf, LevelDev Lc, int bc,
                              const SC* __restrict__ xc, SX* __restrict__ x,
                              const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= Lf.nx || j >= Lf.ny || (done && done[r])) return;
  if (bc == BC_DIRICHLET && on_bnd(i, j, Lf.nx, Lf.ny)) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long id = (long long)j * Lf.nx + i;
  st2(x, r * nf + id, ld2(x, r * nf + id) + interp_bilinear<T, SC>(Lc, xc + r * nc, i, j));
}

// xo = x + dinv .* (f - M x)
template <class T, class SF, class SX, class SO>
__global__ void k_smooth(LevelDev L, int bc, T sre, T sim, VRefE<SF> fin,
                         const SX* __restrict__ x, SO* __restrict__ xo,
                         const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    st2(xo, r * n + id, czero<T>());
    return;
  }
  const SX* xr = x + r * n;
  const C<T> res = ld2(fin.get(), r * n + id) - helm_point<T, SX>(L, bc, sre, sim, xr, i, j);
  st2(xo, r * n + id, cfma(dinv_of<T>(L)[id], res, ld2(xr, id)));
}

// Fused pre-smoothing, residual and restriction for one BX x BY tile of
// coarse nodes: x = dinv .* f on the fine nodes [2I0-2, 2I0+2BX] (+1) held
// in shared memory (the tile's own fine nodes are also written out), then
// f - M x on [2I0-1, 2I0+2BX-1] and its full weighting.  x is computed
// from f where it is needed instead of being read back, so the pair reads
// f once and writes x and the coarse right-hand side once.  Every global
// load a thread needs (D^-1 and f of its x nodes, f and k^2 of its
// residual nodes) is issued up front into registers, so each thread has
// all its loads in flight at once instead of one per loop trip, and the
// residual's operands arrive while the x tile is being built.
template <class T, class SF, class SX, class SC>
__global__ void __launch_bounds__(BX * BY)
k_pre_restrict(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim, VRefE<SF> fin,
               SX* __restrict__ x, SC* __restrict__ fc, const int* __restrict__ done) {
  constexpr int XW = 2 * BX + 3, XH = 2 * BY + 3, RW = 2 * BX + 1, RH = 2 * BY + 1;
  constexpr int NT = BX * BY;
  constexpr int N1 = (XH * XW + NT - 1) / NT, N2 = (RH * RW + NT - 1) / NT;
  __shared__ C<T> xs[XH * XW];
  __shared__ C<T> rsd[RH * RW];
  const int r = blockIdx.z;
  if (done && done[r]) return;
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * BY;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int nfx = Lf.nx, nfy = Lf.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)Lc.nx * Lc.ny;
  const SF* f = fin.get() + r * nf;
  SX* xr = x + r * nf;
  const C<T>* dinv = dinv_of<T>(Lf);
  const T* k2f = k2_of<T>(Lf);
  // operands of the x tile (zero outside the grid and on Dirichlet
  // boundary nodes, where x = 0)
  C<T> dv[N1], fv[N1];
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    const int gi = 2 * I0 - 2 + q % XW, gj = 2 * J0 - 2 + q / XW;
    dv[u] = czero<T>();
    fv[u] = czero<T>();
    if (q < XH * XW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      const long long id = (long long)gj * nfx + gi;
      dv[u] = dinv[id];
      fv[u] = ld2(f, id);
    }
  }
  // operands of the residual nodes
  C<T> f2[N2];
  T k2v[N2];
#pragma unroll
  for (int u = 0; u < N2; ++u) {
    const int q = tid + u * NT;
    const int gi = 2 * I0 - 1 + q % RW, gj = 2 * J0 - 1 + q / RW;
    f2[u] = czero<T>();
    k2v[u] = T(0);
    if (q < RH * RW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      const long long id = (long long)gj * nfx + gi;
      f2[u] = ld2(f, id);
      k2v[u] = k2f[id];
    }
  }
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    if (q < XH * XW) {
      const int gi = 2 * I0 - 2 + q % XW, gj = 2 * J0 - 2 + q / XW;
      const C<T> v = cmul(dv[u], fv[u]);
      if (gi >= 2 * I0 && gi < 2 * I0 + 2 * BX && gi < nfx && gj >= 2 * J0 &&
          gj < 2 * J0 + 2 * BY && gj < nfy)
        st2(xr, (long long)gj * nfx + gi, v);
      xs[q] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < N2; ++u) {
    const int q = tid + u * NT;
    if (q < RH * RW) {
      const int ri = q % RW, rj = q / RW;
      const int gi = 2 * I0 - 1 + ri, gj = 2 * J0 - 1 + rj;
      C<T> v = czero<T>();
      if (gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
          !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
        C<T> cen;
        T cw, ce, cs, cn;
        helm_row<T>(Lf, bc, sre, sim, gi, gj, k2v[u], cen, cw, ce, cs, cn);
        const int c = (rj + 1) * XW + (ri + 1);
        C<T> acc = cmul(cen, xs[c]);
        if (cw != T(0)) acc = rfma(cw, xs[c - 1], acc);
        if (ce != T(0)) acc = rfma(ce, xs[c + 1], acc);
        if (cs != T(0)) acc = rfma(cs, xs[c - XW], acc);
        if (cn != T(0)) acc = rfma(cn, xs[c + XW], acc);
        v = f2[u] - acc;
      }
      rsd[q] = v;
    }
  }
  __syncthreads();
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  if (I >= Lc.nx || J >= Lc.ny) return;
  C<T> acc = czero<T>();
  if (!(bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny))) {
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        const T w = T((2 - abs(a)) * (2 - abs(b))) * T(0.0625);
        acc = rfma(w, rsd[(2 * threadIdx.y + 1 + b) * RW + 2 * threadIdx.x + 1 + a], acc);
      }
  }
  st2(fc, r * nc + (long long)J * Lc.nx + I, acc);
}

// Fused coarse-grid correction and post-smoothing for one BX x BY tile of
// fine nodes: x' = x + P xc on the tile and its 1-node halo in shared
// memory, then xo = x' + dinv .* (f - M x').  x' is never stored.  The
// thread's own f, D^-1 and k^2 are loaded before the tile is built, so
// they arrive while the x' loads are in flight.
template <class T, class SC, class SX, class SF, class SO>
__global__ void __launch_bounds__(BX * BY)
k_prolong_smooth(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim,
                 const SC* __restrict__ xc, const SX* __restrict__ x, VRefE<SF> fin,
                 SO* __restrict__ xo, const int* __restrict__ done) {
  constexpr int PW = BX + 2, PH = BY + 2, NT = BX * BY;
  constexpr int N1 = (PH * PW + NT - 1) / NT;
  __shared__ C<T> xp[PH * PW];
  const int r = blockIdx.z;
  if (done && done[r]) return;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int nfx = Lf.nx, nfy = Lf.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)Lc.nx * Lc.ny;
  const SX* xr = x + r * nf;
  const SC* xcr = xc + r * nc;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool mine = i < nfx && j < nfy;
  const long long id = (long long)j * nfx + i;
  C<T> fown = czero<T>(), down = czero<T>();
  T k2own = T(0);
  if (mine) {
    fown = ld2(fin.get(), r * nf + id);
    down = dinv_of<T>(Lf)[id];
    k2own = k2_of<T>(Lf)[id];
  }
  C<T> xv[N1];
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    const int gi = i0 - 1 + q % PW, gj = j0 - 1 + q / PW;
    xv[u] = czero<T>();
    if (q < PH * PW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy) {
      xv[u] = ld2(xr, (long long)gj * nfx + gi);
      if (!(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy)))
        xv[u] = xv[u] + interp_bilinear<T, SC>(Lc, xcr, gi, gj);
    }
  }
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    if (q < PH * PW) xp[q] = xv[u];
  }
  __syncthreads();
  if (!mine) return;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nfx, nfy)) {
    st2(xo, r * nf + id, czero<T>());
    return;
  }
  C<T> cen;
  T cw, ce, cs, cn;
  helm_row<T>(Lf, bc, sre, sim, i, j, k2own, cen, cw, ce, cs, cn);
  const int c = (threadIdx.y + 1) * PW + (threadIdx.x + 1);
  C<T> acc = cmul(cen, xp[c]);
  if (cw != T(0)) acc = rfma(cw, xp[c - 1], acc);
  if (ce != T(0)) acc = rfma(ce, xp[c + 1], acc);
  if (cs != T(0)) acc = rfma(cs, xp[c - PW], acc);
  if (cn != T(0)) acc = rfma(cn, xp[c + PW], acc);
  const C<T> res = fown - acc;
  st2(xo, r * nf + id, cfma(down, res, xp[c]));
}

// x = Minv f on the coarsest level (dense inverse built at setup)
template <class T, class SF, class SO>
__global__ void k_dense_mv(int n, const C<T>* __restrict__ minv, VRefE<SF> fin,
                           SO* __restrict__ x, const int* __restrict__ done) {
  extern __shared__ unsigned char smraw[];
  C<T>* fs = reinterpret_cast<C<T>*>(smraw);
  const int r = blockIdx.y;
  if (done && done[r]) return;
  const SF* f = fin.get();
  for (int c = threadIdx.x; c < n; c += blockDim.x) fs[c] = ld2(f, (long long)r * n + c);
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const C<T>* mr = minv + (long long)row * n;
  C<T> acc = czero<T>();
  for (int c = 0; c < n; ++c) acc = cfma(mr[c], fs[c], acc);
  st2(x, (long long)r * n + row, acc);
}

}  // namespace

template <class T, class SF, class SX>
void launch_jacobi0(const LevelDev& L, int bc, VRefE<SF> f, SX* x, int nrhs,
                    const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_jacobi0<T, SF, SX><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, f, x,
                                                                       done);
}
template <class T, class SF, class SX, class SC>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                           VRefE<SF> f, const SX* x, SC* fc, int nrhs,
                           const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_resid_restrict<T, SF, SX, SC><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, f, x, fc, done);
}
template <class T, class SC, class SX>
void launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, int bc, const SC* xc,
                        SX* x, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_prolong_add<T, SC, SX><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, xc, x, done);
}
template <class T, class SF, class SX, class SO>
void launch_smooth(const LevelDev& L, int bc, Shift s, VRefE<SF> f, const SX* x,
                   SO* xo, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_smooth<T, SF, SX, SO><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(
      L, bc, (T)s.re, (T)s.im, f, x, xo, done);
}
template <class T, class SF, class SX, class SC>
void launch_pre_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                         VRefE<SF> f, SX* x, SC* fc, int nrhs, const int* done,
                         cudaStream_t st) {
  HZ_COUNT();
  k_pre_restrict<T, SF, SX, SC><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, f, x, fc, done);
}
template <class T, class SC, class SX, class SF, class SO>
void launch_prolong_smooth(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                           const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                           const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_prolong_smooth<T, SC, SX, SF, SO><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, xc, x, f, xo, done);
}
template <class T, class SF, class SO>
void launch_dense_mv(int n, const C<T>* minv, VRefE<SF> f, SO* x, int nrhs,
                     const int* done, cudaStream_t st) {
  HZ_COUNT();
  const int nt = 128;
  k_dense_mv<T, SF, SO><<<dim3((n + nt - 1) / nt, nrhs), nt, n * sizeof(C<T>), st>>>(
      n, minv, f, x, done);
}

// Instantiations: the plain FP64 and FP32 hierarchies (one storage type), and
// the BF16-storage hierarchy under an FP32 V-cycle whose entry vector and
// result stay FP32.
#define HZ_VC_SAME(T)                                                           \
  template void launch_jacobi0<T, C<T>, C<T>>(const LevelDev&, int, VRef<T>,    \
                                              C<T>*, int, const int*,           \
                                              cudaStream_t);                    \
  template void launch_resid_restrict<T, C<T>, C<T>, C<T>>(                     \
      const LevelDev&, const LevelDev&, int, Shift, VRef<T>, const C<T>*,       \
      C<T>*, int, const int*, cudaStream_t);                                    \
  template void launch_prolong_add<T, C<T>, C<T>>(const LevelDev&,              \
                                                  const LevelDev&, int,         \
                                                  const C<T>*, C<T>*, int,      \
                                                  const int*, cudaStream_t);    \
  template void launch_smooth<T, C<T>, C<T>, C<T>>(const LevelDev&, int, Shift, \
                                                   VRef<T>, const C<T>*, C<T>*, \
                                                   int, const int*,             \
                                                   cudaStream_t);               \
  template void launch_dense_mv<T, C<T>, C<T>>(int, const C<T>*, VRef<T>,       \
                                               C<T>*, int, const int*,          \
                                               cudaStream_t);

HZ_VC_SAME(double)
HZ_VC_SAME(float)

using bf2 = __nv_bfloat162;
template void launch_jacobi0<float, float2, bf2>(const LevelDev&, int, VRefE<float2>,
                                                 bf2*, int, const int*, cudaStream_t);
template void launch_jacobi0<float, bf2, bf2>(const LevelDev&, int, VRefE<bf2>, bf2*,
                                              int, const int*, cudaStream_t);
template void launch_resid_restrict<float, float2, bf2, bf2>(
    const LevelDev&, const LevelDev&, int, Shift, VRefE<float2>, const bf2*, bf2*, int,
    const int*, cudaStream_t);
template void launch_resid_restrict<float, bf2, bf2, bf2>(
    const LevelDev&, const LevelDev&, int, Shift, VRefE<bf2>, const bf2*, bf2*, int,
    const int*, cudaStream_t);
template void launch_prolong_add<float, bf2, bf2>(const LevelDev&, const LevelDev&, int,
                                                  const bf2*, bf2*, int, const int*,
                                                  cudaStream_t);
template void launch_smooth<float, float2, bf2, float2>(const LevelDev&, int, Shift,
                                                        VRefE<float2>, const bf2*,
                                                        float2*, int, const int*,
                                                        cudaStream_t);
template void launch_smooth<float, bf2, bf2, bf2>(const LevelDev&, int, Shift,
                                                  VRefE<bf2>, const bf2*, bf2*, int,
                                                  const int*, cudaStream_t);
template void launch_dense_mv<float, bf2, bf2>(int, const float2*, VRefE<bf2>, bf2*, int,
                                               const int*, cudaStream_t);

#define HZ_VC_FUSED(T, SF, SX, SC, SO)                                          \
  template void launch_pre_restrict<T, SF, SX, SC>(                             \
      const LevelDev&, const LevelDev&, int, Shift, VRefE<SF>, SX*, SC*, int,   \
      const int*, cudaStream_t);                                                \
  template void launch_prolong_smooth<T, SC, SX, SF, SO>(                       \
      const LevelDev&, const LevelDev&, int, Shift, const SC*, const SX*,       \
      VRefE<SF>, SO*, int, const int*, cudaStream_t);
HZ_VC_FUSED(double, double2, double2, double2, double2)
HZ_VC_FUSED(float, float2, float2, float2, float2)
HZ_VC_FUSED(float, float2, bf2, bf2, float2)
HZ_VC_FUSED(float, bf2, bf2, bf2, bf2)

}  // namespace hz
