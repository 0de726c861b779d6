// Adjoint-gradient kernels for J(m) = 1/2 sum_s ||S u_s - d_s||^2 with
// k^2 = omega^2 m, and small bookkeeping kernels.
//
// A is complex symmetric up to the boundary scaling D (1 interior, 1/2 edge,
// 1/4 corner under Sommerfeld rows; D A is symmetric), so A^H = D conj(A) D^-1
// and the adjoint field lam = A^-H S^T r is lam = D conj(x) with
// A x = conj(D^-1 S^T r).  Only the diagonal of A depends on m:
// dA_nn/dm_n = -omega^2 - c_n i omega^2 / (h k_n), c_n = number of Sommerfeld
// sides of node n.  Then dJ/dm_n = -sum_s Re(conj(lam_n) dA_nn/dm_n u_n)
//                                = -sum_s Re(D_n x_n dA_nn/dm_n u_n).
#include "hz_common.cuh"

namespace hz {

namespace {

__device__ __forceinline__ int sides(int i, int j, int nx, int ny) {
  return int(i == 0) + int(i == nx - 1) + int(j == 0) + int(j == ny - 1);
}

__global__ void k_accum_iters(const int* iters, int* total, int* maxv, int nrhs,
                              const int* mask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || (mask && mask[r])) return;
  total[r] += iters[r];
  if (iters[r] > maxv[r]) maxv[r] = iters[r];
}

// adj[r][rec[q]] += conj(res) / D, res = u[r][rec[q]] - d[r][q];
// J += 1/2 |res|^2
__global__ void k_adjoint_source(int nx, int ny, int bc, const double2* u,
                                 const int* rec, int nrec, const double2* d,
                                 double2* adj, double* J) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  __shared__ double red[32];
  double contrib = 0.0;
  if (q < nrec) {
    const long long n = (long long)nx * ny;
    const int node = rec[q];
    const bool valid = node >= 0 && (long long)node < n;
    const int i = valid ? node % nx : 0, j = valid ? node / nx : 0;
    // receivers outside the grid or on Dirichlet boundary nodes record zero
    const bool dir_bnd = !valid || ((bc == BC_DIRICHLET) &&
                         (i == 0 || j == 0 || i == nx - 1 || j == ny - 1));
    const double2 uv = dir_bnd ? make_double2(0.0, 0.0) : u[r * n + node];
    const double2 dv = d[(long long)r * nrec + q];
    const double2 res = make_double2(uv.x - dv.x, uv.y - dv.y);
    contrib = 0.5 * (res.x * res.x + res.y * res.y);
    if (!dir_bnd) {
      double D = 1.0;
      if (bc == BC_SOMMERFELD) {
        const int c = sides(i, j, nx, ny);
        D = (c == 0) ? 1.0 : (c == 1 ? 0.5 : 0.25);
      }
      atomicAdd(&adj[r * n + node].x, res.x / D);
      atomicAdd(&adj[r * n + node].y, -res.y / D);
    }
  }
  for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    atomicAdd(J, t);
  }
}

__global__ void k_image(LevelDev L, int bc, double omega, const double2* u,
                        const double2* x, double* grad, int nrhs) {
  const long long n = (long long)L.nx * L.ny;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % L.nx), j = (int)(e / L.nx);
    const int c = (bc == BC_SOMMERFELD) ? sides(i, j, L.nx, L.ny) : 0;
    if (bc == BC_DIRICHLET && (i == 0 || j == 0 || i == L.nx - 1 || j == L.ny - 1))
      continue;
    const double D = (c == 0) ? 1.0 : (c == 1 ? 0.5 : 0.25);
    const double w2 = omega * omega;
    // dA/dm = -omega^2 - i c omega^2 / (h k)
    const double2 ap = make_double2(-w2, c ? -c * w2 / (L.h * sqrt(L.k2d[e])) : 0.0);
    double s = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      const double2 xv = x[r * n + e], uv = u[r * n + e];
      // Re(D x ap u)
      const double2 xa = make_double2(xv.x * ap.x - xv.y * ap.y, xv.x * ap.y + xv.y * ap.x);
      s += D * (xa.x * uv.x - xa.y * uv.y);
    }
    grad[e] -= s;
  }
}

}  // namespace

void launch_accum_iters(const int* iters, int* total, int* maxv, int nrhs,
                        const int* mask, cudaStream_t st) {
  HZ_COUNT();
  k_accum_iters<<<(nrhs + 127) / 128, 128, 0, st>>>(iters, total, maxv, nrhs, mask);
}

void launch_adjoint_source(int nx, int ny, int bc, const double2* u,
                           const int* rec, int nrec, const double2* d,
                           double2* adj, double* J, int nrhs, cudaStream_t st) {
  HZ_COUNT();
  k_adjoint_source<<<dim3((nrec + 255) / 256, nrhs), 256, 0, st>>>(
      nx, ny, bc, u, rec, nrec, d, adj, J);
}

void launch_image(const LevelDev& L, int bc, double omega, const double2* u,
                  const double2* x, double* grad, int nrhs, cudaStream_t st) {
  HZ_COUNT();
  const long long n = (long long)L.nx * L.ny;
  long long nb = (n + 255) / 256;
  if (nb > 8192) nb = 8192;
  k_image<<<(unsigned)nb, 256, 0, st>>>(L, bc, omega, u, x, grad, nrhs);
}

}  // namespace hz
