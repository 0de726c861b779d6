// Batched Krylov kernels for GMRES / flexible GMRES (Sec. 3.3, Algorithm 1):
// multi-vector dot products against the Arnoldi basis (one read of w, one
// read of each basis vector), deterministic two-pass reductions, multi-axpy,
// norms, Givens updates of the Hessenberg columns and the triangular solve.
// Each right-hand side owns its basis, Hessenberg matrix and stopping state;
// all of them live in device memory so that no launch depends on host data.
#include <cstdlib>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "hz_common.cuh"

namespace hz {

namespace {

constexpr int NT = 256;   // threads per block
constexpr int EPT = 8;    // elements per thread
constexpr int CHUNK = NT * EPT;

template <class T> __device__ __forceinline__ C<T> cvt_to(double2 v);
template <> __device__ __forceinline__ double2 cvt_to<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt_to<float>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 wide(double2 v) { return v; }
__device__ __forceinline__ double2 wide(float2 v) { return make_double2(v.x, v.y); }

__device__ __forceinline__ double2 shfl_down2(double2 v, int o) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, o);
  v.y = __shfl_down_sync(0xffffffffu, v.y, o);
  return v;
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int o) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, o);
  v.y = __shfl_down_sync(0xffffffffu, v.y, o);
  return v;
}

// Basis rows are read in 16-byte groups of W values: 1 FP64 pair, 2 FP32
// pairs or 4 FP16 pairs.  Rows start 16-byte aligned (padded row stride).
template <class SB> struct VW;
template <> struct VW<double2> { static constexpr int w = 1; };
template <> struct VW<float2> { static constexpr int w = 2; };
template <> struct VW<__half2> { static constexpr int w = 4; };

__device__ __forceinline__ void ldgrp(const double2* p, long long g, double2* o) {
  o[0] = p[g];
}
__device__ __forceinline__ void ldgrp(const float2* p, long long g, float2* o) {
  const float4 v = reinterpret_cast<const float4*>(p)[g];
  o[0] = make_float2(v.x, v.y);
  o[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ldgrp(const __half2* p, long long g, float2* o) {
  const uint4 v = reinterpret_cast<const uint4*>(p)[g];
  o[0] = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  o[1] = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  o[2] = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
  o[3] = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
}

// Raw 16-byte group g of a basis row and value U of it in compute precision.
template <class SB>
__device__ __forceinline__ uint4 ldraw(const SB* p, long long g) {
  return reinterpret_cast<const uint4*>(p)[g];
}
template <int U>
__device__ __forceinline__ double2 unpk(const uint4& v, const double2*) {
  return make_double2(__hiloint2double((int)v.y, (int)v.x),
                      __hiloint2double((int)v.w, (int)v.z));
}
template <int U>
__device__ __forceinline__ float2 unpk(const uint4& v, const float2*) {
  return U == 0 ? make_float2(__uint_as_float(v.x), __uint_as_float(v.y))
                : make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
}
template <int U>
__device__ __forceinline__ float2 unpk(const uint4& v, const __half2*) {
  const unsigned w = U == 0 ? v.x : (U == 1 ? v.y : (U == 2 ? v.z : v.w));
  __half2 h;
  memcpy(&h, &w, sizeof(h));
  return __half22float2(h);
}
// compile-time loop: f(integral_constant<U>) for U = 0..N-1
template <int N, int U = 0, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (U < N) {
    f(std::integral_constant<int, U>{});
    static_for<N, U + 1>(f);
  }
}

// Block-wide sum of a double held by every thread (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
  __syncthreads();
  return t;
}

// Warp sum of NV values at once (NV a power of two <= 8): log2(NV) halving
// exchanges leave each lane one value, then plain xor steps finish the sum.
// Returns the sum of value *idx; every lane of a group of 32/NV lanes holds
// the same value.
template <int CNT, class T>
__device__ __forceinline__ void halve(T* v, int lane, int o) {
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int k = 0; k < CNT / 2; ++k) {
    const T send = up ? v[k] : v[k + CNT / 2];
    const T keep = up ? v[k + CNT / 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}
template <int NV, class T>
__device__ __forceinline__ T multi_reduce(T* v, int lane, int* idx) {
  int o = 16, id = 0;
  if constexpr (NV >= 2) {
    halve<NV>(v, lane, 16);
    id += ((lane >> 4) & 1) * (NV / 2);
    o = 8;
  }
  if constexpr (NV >= 4) {
    halve<NV / 2>(v, lane, 8);
    id += ((lane >> 3) & 1) * (NV / 4);
    o = 4;
  }
  if constexpr (NV >= 8) {
    halve<NV / 4>(v, lane, 4);
    id += ((lane >> 2) & 1) * (NV / 8);
    o = 2;
  }
  T s = v[0];
  for (; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  *idx = id;
  return s;
}

constexpr int MDOT_TILE = 32;

// Pass 1 (re-orthogonalisation) with no RHS flagged: true in every thread,
// so that the whole block leaves before walking its tiles.
__device__ __forceinline__ bool no_reorth(const KState& ks, int nrhs, int* flag_s) {
  if (threadIdx.x < 32) {
    int any = 0;
    for (int r = threadIdx.x; r < nrhs; r += 32) any |= ks.reorth[r] && !ks.done[r];
    any = __any_sync(0xffffffffu, any);
    if (threadIdx.x == 0) *flag_s = any;
  }
  __syncthreads();
  return *flag_s == 0;
}

// One (RHS r, chunk blk) tile of k_mdot: w's chunk stays in registers while
// the j+1 basis rows stream through (G rows' loads issued before use).  The
// partial dots of up to four rows at a time are summed over the warp
// together (9 shuffles for 8 values), the warps' sums of MDOT_TILE rows are combined
// after one block barrier, and the staging wred[2][NW][MDOT_TILE] (and red,
// for pass 0's ||w||^2) alternates between its halves (par, flipped after
// every barrier), so that no second barrier is needed before the next rows'
// sums are written.  Returns false (no barrier taken) when the RHS takes no
// part.
template <class T, class SB>
__device__ __forceinline__ bool mdot_tile(const SB* __restrict__ V, long long vstride,
                                          long long rs, const C<T>* __restrict__ w,
                                          long long n, const KState& ks, int pass, int j,
                                          int r, int blk, double2* wred, double* red,
                                          int& par) {
  constexpr int TILE = MDOT_TILE, NW = NT / 32;
  constexpr int W = VW<SB>::w, VPT = EPT / W, G = 16 / VPT;
  constexpr int RB = G < 4 ? G : 4, NV2 = 2 * RB;  // rows per warp reduction
  static_assert(G % RB == 0, "row groups");
  if (ks.done[r] || (pass && !ks.reorth[r])) return false;
  // algorithmic bytes of this RHS: w and basis vectors 0..j, read once
  if (ks.abytes && blk == 0 && threadIdx.x == 0)
    atomicAdd(ks.abytes, (unsigned long long)n * (sizeof(C<T>) + (j + 1) * sizeof(SB)));
  // thread element e(k, u) = blk*CHUNK + (k*NT + tid)*W + u
  const long long g0 = (long long)blk * (CHUNK / W) + threadIdx.x;
  const C<T>* wr = w + r * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  C<T> wv[EPT];
  T wn = T(0);
#pragma unroll
  for (int k = 0; k < VPT; ++k)
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const long long e = (g0 + (long long)k * NT) * W + u;
      wv[k * W + u] = (e < n) ? wr[e] : czero<T>();
      wn += wv[k * W + u].x * wv[k * W + u].x + wv[k * W + u].y * wv[k * W + u].y;
    }
  if (pass == 0) {
    double v = (double)wn;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[par * NW + warp] = v;
  }
  bool first = true;
  for (int t0 = 0; t0 <= j; t0 += TILE) {
    const int tend = min(t0 + TILE, j + 1);
    double2* wh = wred + par * NW * TILE + warp * TILE;
    for (int i0 = t0; i0 < tend; i0 += G) {
      // issue every load of the G basis vectors first (16 per thread)
      uint4 raw[G][VPT];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const SB* vr = V + (long long)(i0 + q) * vstride + r * rs;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const long long g = g0 + (long long)k * NT;
          raw[q][k] = (i0 + q < tend && g * W < n) ? ldraw(vr, g) : make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int q4 = 0; q4 < G; q4 += RB) {
        T d[NV2];
#pragma unroll
        for (int c = 0; c < RB; ++c) {
          C<T> a = czero<T>();
#pragma unroll
          for (int k = 0; k < VPT; ++k) {
            static_for<W>([&](auto U) {
              const C<T> v = unpk<U.value>(raw[q4 + c][k], (const SB*)nullptr);
              const C<T> wk = wv[k * W + U.value];
              a.x += v.x * wk.x + v.y * wk.y;
              a.y += v.x * wk.y - v.y * wk.x;
            });
          }
          d[2 * c] = a.x;
          d[2 * c + 1] = a.y;
        }
        int idx;
        const T sum = multi_reduce<NV2, T>(d, lane, &idx);
        const int row = i0 + q4 + (idx >> 1);
        if ((lane & (32 / NV2 - 1)) == 0 && row < tend) {
          double* dst = reinterpret_cast<double*>(wh + (row - t0)) + (idx & 1);
          *dst = (double)sum;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < tend - t0) {
      const double2* wp = wred + par * NW * TILE;
      double2 sum = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        sum.x += wp[q * TILE + threadIdx.x].x;
        sum.y += wp[q * TILE + threadIdx.x].y;
      }
      ks.part[((long long)r * (ks.m + 1) + t0 + threadIdx.x) * ks.nblk_max + blk] = sum;
    }
    if (first && pass == 0 && threadIdx.x == NT - 1) {
      double t = 0.0;
      for (int q = 0; q < NW; ++q) t += red[par * NW + q];
      ks.wpart[(long long)r * ks.nblk_max + blk] = t;
    }
    first = false;
    par ^= 1;
  }
  return true;
}

// Pass `pass` (0 or 1) of classical Gram-Schmidt: partial dot products
// part[r][i][blk] = sum_{e in blk} conj(V_i[e]) w[e], i = 0..j.  Pass 0 also
// stores the partial ||w||^2 in wpart; pass 1 runs only for the RHS whose
// reorth flag the first pass raised.
template <class T, class SB>
__global__ void __launch_bounds__(NT, 4)
k_mdot(const SB* __restrict__ V, long long vstride, long long rs,
       const C<T>* __restrict__ w, long long n, KState ks, int pass, int nrhs,
       int nblk) {
  __shared__ double2 wred[2 * (NT / 32) * MDOT_TILE];
  __shared__ double red[2 * (NT / 32)];
  __shared__ int anyr;
  if (pass && no_reorth(ks, nrhs, &anyr)) return;
  const int j = *ks.jctr;
  int par = 0;
  // persistent loop over (RHS, chunk) tiles
  for (long long tile = blockIdx.x; tile < (long long)nrhs * nblk; tile += gridDim.x)
    mdot_tile<T, SB>(V, vstride, rs, w, n, ks, pass, j, (int)(tile / nblk),
                     (int)(tile % nblk), wred, red, par);
}

// hcol[r][i] = sum_blk part[r][i][blk]; H[r][i][j] = (pass 0) or += (pass 1)
__global__ void k_reduce_cols(KState ks, int nblk, int pass) {
  const int r = blockIdx.y;
  if (ks.done[r] || (pass && !ks.reorth[r])) return;
  const int j = *ks.jctr;
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i > j) return;
  const double2* p = ks.part + ((long long)r * (ks.m + 1) + i) * ks.nblk_max;
  double2 s = make_double2(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) {
    s.x += p[b].x;
    s.y += p[b].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double2 t = shfl_down2(s, o);
    s.x += t.x;
    s.y += t.y;
  }
  if (lane == 0) {
    ks.hcol[(long long)r * (ks.m + 1) + i] = s;
    double2* hp = ks.H + ((long long)r * (ks.m + 1) + i) * ks.m + j;
    if (pass) {
      double2 t = *hp;
      t.x += s.x;
      t.y += s.y;
      *hp = t;
    } else {
      *hp = s;
    }
  }
}

// One (RHS r, chunk blk) tile of k_maxpy: w's chunk is updated in registers
// across all j+1 basis rows, written once, and its squared norm reduced.
// The coefficients come straight from the (L1-resident) column hcol rather
// than through shared memory, so the only block barrier of a tile is the
// one of the norm reduction, whose per-warp sums alternate between the two
// halves of red[2][NT/32] (par): a warp can write the next tile's sum while
// thread 0 still reads this one's, and cannot get two tiles ahead of it.
// Returns false (no barrier taken) for a tile whose RHS takes no part.
template <class T, class SB>
__device__ __forceinline__ bool maxpy_tile(const SB* __restrict__ V, long long vstride,
                                           long long rs, C<T>* __restrict__ w, long long n,
                                           const KState& ks, int pass, int j, int r,
                                           int blk, double* red, int par) {
  constexpr int W = VW<SB>::w, VPT = EPT / W, G = 16 / VPT;
  if (ks.done[r] || (pass && !ks.reorth[r])) return false;
  // algorithmic bytes of this RHS: read w and basis 0..j, write w
  if (ks.abytes && blk == 0 && threadIdx.x == 0)
    atomicAdd(ks.abytes, (unsigned long long)n * (2 * sizeof(C<T>) + (j + 1) * sizeof(SB)));
  const long long g0 = (long long)blk * (CHUNK / W) + threadIdx.x;
  C<T>* wr = w + r * n;
  const double2* hc = ks.hcol + (long long)r * (ks.m + 1);
  C<T> acc[EPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k)
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const long long e = (g0 + (long long)k * NT) * W + u;
      acc[k * W + u] = (e < n) ? wr[e] : czero<T>();
    }
  for (int q0 = 0; q0 <= j; q0 += G) {
    uint4 raw[G][VPT];
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const SB* vr = V + (long long)(q0 + q) * vstride + r * rs;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const long long g = g0 + (long long)k * NT;
        raw[q][k] = (q0 + q <= j && g * W < n) ? ldraw(vr, g) : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const C<T> h = (q0 + q <= j) ? cvt_to<T>(hc[q0 + q]) : czero<T>();
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        static_for<W>([&](auto U) {
          const C<T> v = unpk<U.value>(raw[q][k], (const SB*)nullptr);
          acc[k * W + U.value].x -= v.x * h.x - v.y * h.y;
          acc[k * W + U.value].y -= v.x * h.y + v.y * h.x;
        });
      }
    }
  }
  T wn = T(0);
#pragma unroll
  for (int k = 0; k < VPT; ++k)
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const long long e = (g0 + (long long)k * NT) * W + u;
      if (e < n) {
        wr[e] = acc[k * W + u];
        wn += acc[k * W + u].x * acc[k * W + u].x + acc[k * W + u].y * acc[k * W + u].y;
      }
    }
  double v = (double)wn;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  double* rp = red + par * (NT / 32);
  if ((threadIdx.x & 31) == 0) rp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < NT / 32; ++q) t += rp[q];
    ks.npart[(long long)r * ks.nblk_max + blk] = t;
  }
  return true;
}

// w -= sum_{i<=j} V_i hcol_i, and the partial ||w||^2 of the result in npart
template <class T, class SB>
__global__ void __launch_bounds__(NT, 4)
k_maxpy(const SB* __restrict__ V, long long vstride, long long rs,
        C<T>* __restrict__ w, long long n, KState ks, int pass, int nrhs, int nblk) {
  __shared__ double red[2 * (NT / 32)];
  __shared__ int anyr;
  if (pass && no_reorth(ks, nrhs, &anyr)) return;
  const int j = *ks.jctr;
  int par = 0;
  for (long long tile = blockIdx.x; tile < (long long)nrhs * nblk; tile += gridDim.x)
    if (maxpy_tile<T, SB>(V, vstride, rs, w, n, ks, pass, j, (int)(tile / nblk),
                          (int)(tile % nblk), red, par))
      par ^= 1;
}

// The same two kernels over the tiles of several grids (GroupDesc).
template <class T, class SB>
__global__ void __launch_bounds__(NT)
k_mdot_group(const __grid_constant__ GroupDesc gd, int pass) {
  __shared__ double2 wred[2 * (NT / 32) * MDOT_TILE];
  __shared__ double red[2 * (NT / 32)];
  const long long total = gd.start[gd.count];
  int par = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int g = 0;
    while (tile >= gd.start[g + 1]) ++g;
    const GroupMember& M = gd.m[g];
    const long long lt = tile - gd.start[g];
    mdot_tile<T, SB>((const SB*)M.V, M.vstride, M.rs, (const C<T>*)M.w, M.n, M.ks, pass,
                     *M.ks.jctr, (int)(lt / M.nblk), (int)(lt % M.nblk), wred, red, par);
  }
}

template <class T, class SB>
__global__ void __launch_bounds__(NT)
k_maxpy_group(const __grid_constant__ GroupDesc gd, int pass) {
  __shared__ double red[2 * (NT / 32)];
  const long long total = gd.start[gd.count];
  int par = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int g = 0;
    while (tile >= gd.start[g + 1]) ++g;
    const GroupMember& M = gd.m[g];
    const long long lt = tile - gd.start[g];
    if (maxpy_tile<T, SB>((const SB*)M.V, M.vstride, M.rs, (C<T>*)M.w, M.n, M.ks, pass,
                          *M.ks.jctr, (int)(lt / M.nblk), (int)(lt % M.nblk), red, par))
      par ^= 1;
  }
}

// ---------------------------------------------------------------------------
// TMA-pipelined Gram-Schmidt kernels.  One producer warp streams chunks of
// basis rows (CHUNK values of G consecutive basis vectors of one RHS, 32 KB
// per stage) from HBM into a ring of shared-memory stages with bulk copies
// (cp.async.bulk) completing on mbarriers; NCW consumer warps read each
// stage from shared memory.  The bytes in flight per SM are set by the ring
// (NSTAGE x 32 KB), not by registers, and the next tile's chunk of w is
// prefetched into registers while the current tile streams.  Every wait is
// bounded: after KState::wait_ns (kWaitNs) the kernel raises ks.fault, stops waiting and
// still takes part in every block barrier, so the launch always ends; the
// host reports the flag.
constexpr int NSTAGE = 6;
constexpr int STAGE_BYTES = 32768;
constexpr int RING_BYTES = NSTAGE * STAGE_BYTES;
constexpr unsigned long long kWaitNs = 2000000000ull;

template <class SB, int NTC> struct Cgs {
  static constexpr int W = VW<SB>::w;                          // values per 16 B
  static constexpr int ROWB = CHUNK * (int)sizeof(SB);         // bytes per row chunk
  static constexpr int G = STAGE_BYTES / ROWB;                 // vectors per stage
  static constexpr int VPT = CHUNK / (NTC * W);                // groups per thread
  static_assert(VPT >= 1 && VPT * NTC * W == CHUNK, "chunk split");
};

__device__ __forceinline__ unsigned sm_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(sm_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` of barrier b; false after limit ns
// (KState::wait_ns: kWaitNs unless a fault drill shortened it).
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          unsigned long long limit) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    for (int k = 0; k < 64; ++k)
      if (mbar_test(b, parity)) return true;
    if (gtimer() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
      "[%3];" ::"r"(sm_addr(dst)),
      "l"(src), "r"(bytes), "r"(sm_addr(b))
      : "memory");
}
// named barrier of the NTC consumer threads only
template <int NTC>
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NTC) : "memory");
}


// RHS that take part in this pass, compacted into act[] by warp 0.
__device__ __forceinline__ void active_rhs(const KState& ks, int pass, int nrhs,
                                           int* act, int* nact) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int cnt = 0;
  for (int base = 0; base < nrhs; base += 32) {
    const int r = base + lane;
    const bool a = r < nrhs && !ks.done[r] && (!pass || ks.reorth[r]);
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (a) act[cnt + __popc(m & ((1u << lane) - 1u))] = r;
    cnt += __popc(m);
  }
  if (lane == 0) *nact = cnt;
}

// Producer side of one stage: row chunk blk of vectors i0 .. i0+nv-1 of RHS r.
template <class SB>
__device__ __forceinline__ void produce(unsigned char* stage, unsigned long long* full,
                                        const SB* V, long long vstride, long long rs,
                                        int r, int blk, int i0, int nv) {
  constexpr int ROWB = CHUNK * (int)sizeof(SB);
  const long long off = (long long)blk * CHUNK;
  const long long cnt = (rs - off < CHUNK) ? (rs - off) : CHUNK;
  const unsigned bytes = (unsigned)(cnt * (long long)sizeof(SB));
  mbar_expect_tx(full, bytes * (unsigned)nv);
  for (int q = 0; q < nv; ++q)
    bulk_g2s(stage + q * ROWB, V + (long long)(i0 + q) * vstride + r * rs + off, bytes,
             full);
}

// Chunk blk of RHS row w_r into registers: value k*W+u of this consumer
// thread is element blk*CHUNK + (k*NTC + tid)*W + u (zero beyond n).
template <class T, int W, int VPT, int NTC>
__device__ __forceinline__ void load_chunk(C<T>* dst, const C<T>* wr, long long off,
                                           long long n) {
#pragma unroll
  for (int k = 0; k < VPT; ++k)
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const long long e = off + (long long)(k * NTC + threadIdx.x) * W + u;
      dst[k * W + u] = (e < n) ? wr[e] : czero<T>();
    }
}

// Ring slot of one item: stage s (0 .. NSTAGE-1) and the parity of its use.
struct Slot {
  int s = 0;
  unsigned ph = 0;
  __device__ __forceinline__ void next() {
    if (++s == NSTAGE) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Producer lane: wait until the consumers released the stage of slot q.
__device__ __forceinline__ bool producer_acquire(unsigned long long* empty, Slot q,
                                                 volatile int* s_abort, int* fault,
                                                 unsigned long long limit) {
  if (*s_abort || !mbar_wait(&empty[q.s], q.ph ^ 1u, limit)) {
    *s_abort = 1;
    atomicExch(fault, 1);
    return false;
  }
  return true;
}
// No bulk copy may still be landing when the block exits: wait for the last
// min(issued, NSTAGE) stages (slot `at` is the one after the last issued).
__device__ __forceinline__ void producer_drain(unsigned long long* full, long long issued,
                                               Slot at, int* fault, unsigned long long limit) {
  const int cnt = issued < NSTAGE ? (int)issued : NSTAGE;
  for (int u = 0; u < cnt; ++u) {
    // step back one slot
    if (at.s == 0) {
      at.s = NSTAGE - 1;
      at.ph ^= 1u;
    } else {
      --at.s;
    }
    if (!mbar_wait(&full[at.s], at.ph, limit)) atomicExch(fault, 1);
  }
}
__device__ __forceinline__ bool consumer_acquire(unsigned long long* full, Slot q,
                                                 volatile int* s_abort, int* fault,
                                                 unsigned long long limit) {
  if (*s_abort || !mbar_wait(&full[q.s], q.ph, limit)) {
    *s_abort = 1;
    atomicExch(fault, 1);
    return false;
  }
  return true;
}
__device__ __forceinline__ void consumer_release(unsigned long long* empty, Slot q) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[q.s]);
}

template <int NCW>
__device__ __forceinline__ void ring_init(unsigned long long* full,
                                          unsigned long long* empty,
                                          volatile int* s_abort) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// Position of a work item of k_mdot_tma: active RHS a, row chunk blk,
// vector group grp; advanced without divisions.
struct Item {
  int a, blk, grp;
  __device__ __forceinline__ void next(int nblk, int ngrp) {
    if (++grp == ngrp) {
      grp = 0;
      if (++blk == nblk) {
        blk = 0;
        ++a;
      }
    }
  }
};

// Pass `pass` of classical Gram-Schmidt (same contract as k_mdot).  The
// work items (RHS, row chunk, group of G vectors) of all active RHS are
// split evenly over the blocks, so every block streams the same number of
// bytes whatever j and the number of converged RHS.  The per-warp sums of
// FLUSH items are combined across warps after one consumer barrier; the
// staging buffers alternate between two halves, so the next items' sums go
// to the other half while this half is read, and the barrier of the next
// flush orders this half's reads before its next writes.
template <class T, class SB, int NCW>
__global__ void __launch_bounds__(32 * NCW + 32, 1)
k_mdot_tma(const SB* __restrict__ V, long long vstride, long long rs,
           const C<T>* __restrict__ w, long long n, KState ks, int pass, int nrhs,
           int nblk) {
  constexpr int NTC = 32 * NCW;
  using P = Cgs<SB, NTC>;
  constexpr int W = P::W, G = P::G, VPT = P::VPT, NV = 2 * G, E = VPT * W;
  constexpr int FLUSH = 32 / G;   // items per reduction flush
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ unsigned long long full[NSTAGE], empty[NSTAGE];
  __shared__ int act[1024];
  __shared__ int s_nact;
  __shared__ volatile int s_abort;
  __shared__ double wred[2][NCW][2 * 32];
  __shared__ double wnred[2][NCW][FLUSH];
  __shared__ int3 pitem[2][FLUSH];   // (RHS, chunk, group) of the pending items
  const int j = *ks.jctr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  active_rhs(ks, pass, nrhs, act, &s_nact);
  ring_init<NCW>(full, empty, &s_abort);
  __syncthreads();
  const int ngrp = (j + 1 + G - 1) / G;
  const long long items = (long long)s_nact * nblk * ngrp;
  const long long lo = items * blockIdx.x / gridDim.x;
  const long long hi = items * (blockIdx.x + 1) / gridDim.x;
  const int nitems = (int)(hi - lo);
  Item it0;
  {
    const long long tile = lo / ngrp;
    it0.grp = (int)(lo - tile * ngrp);
    it0.a = (int)(tile / nblk);
    it0.blk = (int)(tile - (long long)it0.a * nblk);
  }

  if (warp == NCW) {  // producer (a fault drill's starve mode issues nothing)
    if (lane == 0 && !ks.starve) {
      Slot sl;
      Item it = it0;
      int t = 0;
      for (; t < nitems; ++t) {
        if (!producer_acquire(empty, sl, &s_abort, ks.fault, ks.wait_ns)) break;
        const int i0 = it.grp * G, nv = min(G, j + 1 - i0);
        produce<SB>(stages + sl.s * STAGE_BYTES, &full[sl.s], V, vstride, rs, act[it.a],
                    it.blk, i0, nv);
        sl.next();
        it.next(nblk, ngrp);
      }
      producer_drain(full, t, sl, ks.fault, ks.wait_ns);
    }
  } else {  // consumers
    int cur_a = -1, cur_blk = -1;
    bool have_next = false;
    C<T> wv[E], wq[E];
    int pend = 0, buf = 0;
    Slot sl;
    Item it = it0;
    for (int t = 0; t < nitems; ++t) {
      const long long off = (long long)it.blk * CHUNK;
      if (it.a != cur_a || it.blk != cur_blk) {
        if (have_next) {
#pragma unroll
          for (int e = 0; e < E; ++e) wv[e] = wq[e];
        } else {
          load_chunk<T, W, VPT, NTC>(wv, w + act[it.a] * n, off, n);
        }
        cur_a = it.a;
        cur_blk = it.blk;
        // prefetch the chunk of w of the next tile if this block reaches it
        const int left = nitems - t - (ngrp - it.grp);   // items after this tile
        int na = it.a, nb = it.blk + 1;
        if (nb == nblk) {
          nb = 0;
          ++na;
        }
        have_next = left > 0;
        if (have_next)
          load_chunk<T, W, VPT, NTC>(wq, w + act[na] * n, (long long)nb * CHUNK, n);
        if (pass == 0 && it.grp == 0) {
          T wn = T(0);
#pragma unroll
          for (int e = 0; e < E; ++e) wn += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
          for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
          if (lane == 0) wnred[buf][warp][pend] = (double)wn;
        }
      }
      if (threadIdx.x == 0) pitem[buf][pend] = make_int3(it.a, it.blk, it.grp);
      T acc[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) acc[c] = T(0);
      if (consumer_acquire(full, sl, &s_abort, ks.fault, ks.wait_ns)) {
        const int nv = min(G, j + 1 - it.grp * G);
        const long long valid = n - off;   // values of this chunk inside the row
        const unsigned char* sb = stages + sl.s * STAGE_BYTES;
        // FULL: all G vectors of the group exist and the chunk lies inside
        // the row, so no value needs a bounds test
        auto dot = [&](auto FULL) {
#pragma unroll
          for (int qq = 0; qq < G; ++qq) {
            if (FULL.value || qq < nv) {
#pragma unroll
              for (int k = 0; k < VPT; ++k) {
                const int g = k * NTC + threadIdx.x;
                if (FULL.value || (long long)g * W < valid) {
                  const uint4 raw =
                      *reinterpret_cast<const uint4*>(sb + qq * P::ROWB + g * 16);
                  static_for<W>([&](auto U) {
                    const C<T> v = unpk<U.value>(raw, (const SB*)nullptr);
                    const C<T> wk = wv[k * W + U.value];
                    acc[2 * qq] += v.x * wk.x + v.y * wk.y;
                    acc[2 * qq + 1] += v.x * wk.y - v.y * wk.x;
                  });
                }
              }
            }
          }
        };
        if (nv == G && valid >= CHUNK)
          dot(std::true_type{});
        else
          dot(std::false_type{});
      }
      consumer_release(empty, sl);
      sl.next();
      int idx = 0;
      const T sum = multi_reduce<NV>(acc, lane, &idx);
      if ((lane & (32 / NV - 1)) == 0) wred[buf][warp][pend * NV + idx] = (double)sum;
      ++pend;
      it.next(nblk, ngrp);
      if (pend == FLUSH || t + 1 == nitems) {
        consumers_sync<NTC>();
        const int v = threadIdx.x;
        if (v < pend * G) {
          const int3 pi = pitem[buf][v / G];
          const int i = pi.z * G + v % G;
          if (i <= j) {
            double2 sm = make_double2(0.0, 0.0);
#pragma unroll
            for (int ww = 0; ww < NCW; ++ww) {
              sm.x += wred[buf][ww][2 * v];
              sm.y += wred[buf][ww][2 * v + 1];
            }
            ks.part[((long long)act[pi.x] * (ks.m + 1) + i) * ks.nblk_max + pi.y] = sm;
          }
        }
        if (pass == 0 && v < pend) {
          const int3 pi = pitem[buf][v];
          if (pi.z == 0) {
            double tw = 0.0;
#pragma unroll
            for (int ww = 0; ww < NCW; ++ww) tw += wnred[buf][ww][v];
            ks.wpart[(long long)act[pi.x] * ks.nblk_max + pi.y] = tw;
          }
        }
        buf ^= 1;
        pend = 0;
      }
    }
    if (ks.abytes && threadIdx.x == 0 && nitems > 0) {
      // algorithmic bytes: each basis row chunk once, w once per chunk
      // (counted by the block that holds the chunk's first group)
      unsigned long long b = 0;
      Item q = it0;
      for (int t = 0; t < nitems; ++t) {
        const long long off = (long long)q.blk * CHUNK;
        const long long vals = (n - off < CHUNK) ? (n - off) : CHUNK;
        b += (unsigned long long)vals * (min(G, j + 1 - q.grp * G) * sizeof(SB) +
                                         (q.grp == 0 ? sizeof(C<T>) : 0));
        q.next(nblk, ngrp);
      }
      atomicAdd(ks.abytes, b);
    }
  }
  __syncthreads();
}

// w -= sum_{i<=j} V_i hcol_i and the partial ||w||^2 (same contract as
// k_maxpy).  Blocks take whole (RHS, chunk) tiles round-robin, since the
// chunk of w is updated in registers across all j+1 vectors.
template <class T, class SB, int NCW>
__global__ void __launch_bounds__(32 * NCW + 32, 1)
k_maxpy_tma(const SB* __restrict__ V, long long vstride, long long rs,
            C<T>* __restrict__ w, long long n, KState ks, int pass, int nrhs, int nblk) {
  constexpr int NTC = 32 * NCW;
  using P = Cgs<SB, NTC>;
  constexpr int W = P::W, G = P::G, VPT = P::VPT, E = VPT * W;
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ unsigned long long full[NSTAGE], empty[NSTAGE];
  __shared__ int act[1024];
  __shared__ int s_nact;
  __shared__ volatile int s_abort;
  __shared__ double red[NCW];
  const int j = *ks.jctr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  active_rhs(ks, pass, nrhs, act, &s_nact);
  ring_init<NCW>(full, empty, &s_abort);
  __syncthreads();
  const int ngrp = (j + 1 + G - 1) / G;
  const int tiles = s_nact * nblk;

  if (warp == NCW) {  // producer (a fault drill's starve mode issues nothing)
    if (lane == 0 && !ks.starve) {
      Slot sl;
      long long t = 0;
      bool stop = false;
      for (int tile = blockIdx.x; tile < tiles && !stop; tile += gridDim.x) {
        const int a = tile / nblk, blk = tile - a * nblk;
        for (int grp = 0; grp < ngrp; ++grp, ++t) {
          if (!producer_acquire(empty, sl, &s_abort, ks.fault, ks.wait_ns)) {
            stop = true;
            break;
          }
          produce<SB>(stages + sl.s * STAGE_BYTES, &full[sl.s], V, vstride, rs, act[a],
                      blk, grp * G, min(G, j + 1 - grp * G));
          sl.next();
        }
      }
      producer_drain(full, t, sl, ks.fault, ks.wait_ns);
    }
  } else {  // consumers
    Slot sl;
    unsigned long long bytes = 0;
    C<T> acc[E], nxt[E];
    bool have_next = false;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int a = tile / nblk, blk = tile - a * nblk;
      const int r = act[a];
      const long long off = (long long)blk * CHUNK;
      const long long valid = n - off;
      C<T>* wr = w + r * n;
      if (have_next) {
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = nxt[e];
      } else {
        load_chunk<T, W, VPT, NTC>(acc, wr, off, n);
      }
      // prefetch the next tile's chunk of w (a different chunk: no overlap
      // with the stores of this tile)
      const int nt = tile + gridDim.x;
      have_next = nt < tiles;
      if (have_next) {
        const int na = nt / nblk;
        load_chunk<T, W, VPT, NTC>(nxt, w + act[na] * n, (long long)(nt - na * nblk) * CHUNK,
                                   n);
      }
      const double2* hc = ks.hcol + (long long)r * (ks.m + 1);
      for (int grp = 0; grp < ngrp; ++grp) {
        const int nv = min(G, j + 1 - grp * G);
        C<T> h[G];
#pragma unroll
        for (int qq = 0; qq < G; ++qq)
          h[qq] = (qq < nv) ? cvt_to<T>(hc[grp * G + qq]) : czero<T>();
        if (consumer_acquire(full, sl, &s_abort, ks.fault, ks.wait_ns)) {
          const unsigned char* sb = stages + sl.s * STAGE_BYTES;
#pragma unroll
          for (int qq = 0; qq < G; ++qq) {
            if (qq < nv) {
#pragma unroll
              for (int k = 0; k < VPT; ++k) {
                const int g = k * NTC + threadIdx.x;
                if ((long long)g * W < valid) {
                  const uint4 raw =
                      *reinterpret_cast<const uint4*>(sb + qq * P::ROWB + g * 16);
                  static_for<W>([&](auto U) {
                    const C<T> v = unpk<U.value>(raw, (const SB*)nullptr);
                    acc[k * W + U.value].x -= v.x * h[qq].x - v.y * h[qq].y;
                    acc[k * W + U.value].y -= v.x * h[qq].y + v.y * h[qq].x;
                  });
                }
              }
            }
          }
        }
        consumer_release(empty, sl);
        sl.next();
      }
      T wn = T(0);
#pragma unroll
      for (int k = 0; k < VPT; ++k)
#pragma unroll
        for (int u = 0; u < W; ++u) {
          const long long e = off + (long long)(k * NTC + threadIdx.x) * W + u;
          if (e < n) {
            wr[e] = acc[k * W + u];
            wn += acc[k * W + u].x * acc[k * W + u].x + acc[k * W + u].y * acc[k * W + u].y;
          }
        }
      double d = (double)wn;
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) red[warp] = d;
      consumers_sync<NTC>();
      if (threadIdx.x == 0) {
        double tsum = 0.0;
#pragma unroll
        for (int ww = 0; ww < NCW; ++ww) tsum += red[ww];
        ks.npart[(long long)r * ks.nblk_max + blk] = tsum;
      }
      consumers_sync<NTC>();
      const long long vals = valid < CHUNK ? valid : CHUNK;
      bytes += (unsigned long long)vals * (2 * sizeof(C<T>) + (j + 1) * sizeof(SB));
    }
    if (ks.abytes && threadIdx.x == 0 && bytes) atomicAdd(ks.abytes, bytes);
  }
  __syncthreads();
}

// After the first pass: ||w|| (wpart) and ||w - V h|| (npart) per RHS; the
// second pass runs only where the first cancelled more than a factor 1/eta
// (Kahan-Parlett "twice is enough" test).  hnorm = ||w - V h||.
__global__ void k_reorth_decide(KState ks, int nblk, double eta) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  if (ks.done[r]) {
    if (threadIdx.x == 0) ks.reorth[r] = 0;
    return;
  }
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    a += ks.wpart[(long long)r * ks.nblk_max + q];
    b += ks.npart[(long long)r * ks.nblk_max + q];
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    const double nw = sqrt(a), nw1 = sqrt(b);
    ks.hnorm[r] = nw1;
    ks.reorth[r] = (nw1 < eta * nw) ? 1 : 0;
  }
}

template <class T>
__global__ void __launch_bounds__(NT)
k_norm2_part(VRef<T> w, long long n, KState ks, const int* __restrict__ done) {
  __shared__ double red[NT / 32];
  const int r = blockIdx.y;
  if (done && done[r]) return;
  const long long base = (long long)blockIdx.x * CHUNK + threadIdx.x;
  const C<T>* wr = w.get() + r * n;
  T s = T(0);
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const long long e = base + k * NT;
    if (e < n) {
      const C<T> v = wr[e];
      s += v.x * v.x + v.y * v.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < NT / 32; ++q) t += red[q];
    ks.npart[(long long)r * ks.nblk_max + blockIdx.x] = t;
  }
}

__global__ void k_reduce_norm(KState ks, int nblk, double* out, int sqrt_it) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    s += ks.npart[(long long)r * ks.nblk_max + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
    out[r] = sqrt_it ? sqrt(t) : t;
  }
}

// status codes mirrored from hz.h
enum { ST_OK = 0, ST_NOT_CONVERGED = 4, ST_BREAKDOWN = 5, ST_NAN = 6 };

__global__ void k_krylov_init(KState ks, int nrhs, const int* done_in,
                              const double* bnorm_src, double tol) {
  const int r = threadIdx.x;
  int d = 1;
  if (r < nrhs) {
    d = done_in ? done_in[r] : 0;
    const double b = ks.beta[r];
    const double bn = bnorm_src ? bnorm_src[r] : b;
    ks.bnorm[r] = bn;
    ks.iters[r] = 0;
    if (!d) ks.stat[r] = ST_OK;   // an RHS that stopped keeps its status
    ks.g[(long long)r * (ks.m + 1)] = make_double2(b, 0.0);
    ks.hnorm[r] = b;
    if (!d) {
      if (!isfinite(b)) {
        d = 1;
        ks.stat[r] = ST_NAN;
      } else if (b == 0.0 || b <= tol * bn) {
        d = 1;
      }
    }
    ks.done[r] = d;
  }
  const int all = __syncthreads_and(d);
  if (r == 0) {
    *ks.jctr = 0;
    *ks.alldone = all;
  }
}

template <class T, class SB>
__global__ void __launch_bounds__(256)
k_scale_into(VRef<T> w, VRefE<SB> out, long long rs, const double* __restrict__ s,
             long long n, const int* __restrict__ done, C<T>* __restrict__ copy) {
  constexpr int U = 4;   // values per thread and trip: one 16-byte FP16 group
  const int r = blockIdx.y;
  if (done && done[r]) return;
  // one FP64 reciprocal per block (FP64 division is slow on this GPU)
  __shared__ T f_s;
  if (threadIdx.x == 0) {
    const double sv = s[r];
    f_s = (sv != 0.0) ? T(1.0 / sv) : T(0);
  }
  __syncthreads();
  const T f = f_s;
  const C<T>* wr = w.get() + r * n;
  SB* orow = out.get() + r * rs;
  C<T>* crow = copy ? copy + r * n : nullptr;
  // rows of the basis are padded to rs >= n (a multiple of 4), so groups of
  // U values start 16-byte aligned in the FP16 basis; the padding is written
  // as zero (group loads read it)
  for (long long e0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * U; e0 < rs;
       e0 += (long long)gridDim.x * blockDim.x * U) {
    C<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = (e0 + u < n) ? wr[e0 + u] : czero<T>();
    SB sv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) st2(sv, u, f * v[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u < rs) orow[e0 + u] = sv[u];
    // the stored (rounded) value, also kept in compute precision as the
    // V-cycle's input of the next step
    if (crow) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e0 + u < n) crow[e0 + u] = ld2(sv, u);
    }
  }
}

// Apply the previous rotations to column j, build the rotation that
// annihilates h_{j+1,j}, update the least-squares right-hand side g and
// decide convergence (|g_{j+1}| <= tol ||b||), breakdown, NaN or the cap.
// One block per RHS: the column is staged in shared memory so the
// sequential rotation chain runs out of shared memory, not DRAM.
__global__ void k_givens(KState ks, double tol, int maxit) {
  extern __shared__ unsigned char smraw[];
  double2* col = reinterpret_cast<double2*>(smraw);   // j + 2 entries
  const int r = blockIdx.x;
  if (ks.done[r]) return;
  const int j = *ks.jctr;
  const int m = ks.m;
  double2* Hc = ks.H + (long long)r * (m + 1) * m + j;  // H[r][i][j] = Hc[i*m]
  // the previous rotations are staged too, so the sequential chain below
  // reads shared memory only
  double2* sn = col + (m + 2);                                  // j entries
  double* cs = reinterpret_cast<double*>(sn + m);               // j entries
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = Hc[(long long)i * m];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs[i] = ks.cs[(long long)r * m + i];
    sn[i] = ks.sn[(long long)r * m + i];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double2 a = col[0];
  for (int i = 0; i < j; ++i) {
    const double2 b = col[i + 1];
    const double c = cs[i];
    const double2 sv = sn[i];
    // t = c a + s b ; b' = -conj(s) a + c b
    col[i] = make_double2(c * a.x + (sv.x * b.x - sv.y * b.y),
                          c * a.y + (sv.x * b.y + sv.y * b.x));
    a = make_double2(-(sv.x * a.x + sv.y * a.y) + c * b.x,
                     -(sv.x * a.y - sv.y * a.x) + c * b.y);
  }
  const double hb = ks.hnorm[r];
  const double am = sqrt(a.x * a.x + a.y * a.y);
  double c;
  double2 sv;
  if (hb == 0.0) {
    c = 1.0;
    sv = make_double2(0.0, 0.0);
  } else if (am == 0.0) {
    c = 0.0;
    sv = make_double2(1.0, 0.0);
  } else {
    const double t = sqrt(am * am + hb * hb);
    c = am / t;
    sv = make_double2(a.x / am * hb / t, a.y / am * hb / t);
  }
  ks.cs[(long long)r * m + j] = c;
  ks.sn[(long long)r * m + j] = sv;
  col[j] = make_double2(c * a.x + sv.x * hb, c * a.y + sv.y * hb);
  for (int i = 0; i <= j; ++i) Hc[(long long)i * m] = col[i];
  Hc[(long long)(j + 1) * m] = make_double2(0.0, 0.0);
  double2* g = ks.g + (long long)r * (m + 1);
  const double2 gj = g[j];
  const double2 g1 = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
  g[j + 1] = g1;
  g[j] = make_double2(c * gj.x, c * gj.y);
  const double res = sqrt(g1.x * g1.x + g1.y * g1.y);
  ks.iters[r] = j + 1;
  int d = 0;
  if (!isfinite(res) || !isfinite(hb)) {
    d = 1;
    ks.stat[r] = ST_NAN;
  } else if (res <= tol * ks.bnorm[r]) {
    d = 1;
  } else if (hb == 0.0) {
    d = 1;
    ks.stat[r] = ST_BREAKDOWN;
  } else if (j + 1 >= maxit) {
    d = 1;
    ks.stat[r] = ST_NOT_CONVERGED;
  }
  ks.done[r] = d;
}

// All RHS done?  Otherwise advance the Arnoldi column counter.
__global__ void k_givens_finish(KState ks, int nrhs) {
  const int r = threadIdx.x;
  const int d = (r < nrhs) ? ks.done[r] : 1;
  const int all = __syncthreads_and(d);
  if (r == 0) {
    *ks.alldone = all;
    if (!all) *ks.jctr = *ks.jctr + 1;
  }
}

// Back substitution R y = g for each RHS (R = rotated Hessenberg), one block
// per RHS: the right-hand side lives in shared memory and each step updates
// the rows above the pivot in parallel.
__global__ void k_trisolve(KState ks) {
  extern __shared__ unsigned char smraw[];
  double2* gs = reinterpret_cast<double2*>(smraw);   // k entries
  __shared__ double2 yi_s;
  const int r = blockIdx.x;
  const int m = ks.m, k = ks.iters[r];
  const double2* H = ks.H + (long long)r * (m + 1) * m;
  double2* y = ks.y + (long long)r * m;
  for (int q = threadIdx.x; q < k; q += blockDim.x) gs[q] = ks.g[(long long)r * (m + 1) + q];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double2 d = H[(long long)i * m + i], s = gs[i];
      const double dm = d.x * d.x + d.y * d.y;
      const double2 v = (dm > 0.0) ? make_double2((s.x * d.x + s.y * d.y) / dm,
                                                  (s.y * d.x - s.x * d.y) / dm)
                                   : make_double2(0.0, 0.0);
      y[i] = v;
      yi_s = v;
    }
    __syncthreads();
    const double2 yv = yi_s;
    for (int q = threadIdx.x; q < i; q += blockDim.x) {
      const double2 h = H[(long long)q * m + i];
      gs[q].x -= h.x * yv.x - h.y * yv.y;
      gs[q].y -= h.x * yv.y + h.y * yv.x;
    }
    __syncthreads();
  }
}

// x (+)= sum_{i < iters} y_i V_i.  Same tiling as k_maxpy: each block
// takes (RHS, chunk) tiles round-robin, keeps the chunk of x in registers,
// streams the basis rows in 16-byte groups with G rows' loads issued before
// use, and reads y straight from its L1-resident column (no barrier).
template <class SB, class Tx>
__global__ void __launch_bounds__(NT, 4)
k_update(const SB* __restrict__ V, long long vstride, long long rs, KState ks,
         C<Tx>* __restrict__ x, int accumulate, long long n, int nrhs, int nblk) {
  constexpr int W = VW<SB>::w, VPT = EPT / W, G = 16 / VPT;
  for (long long tile = blockIdx.x; tile < (long long)nrhs * nblk; tile += gridDim.x) {
    const int r = (int)(tile / nblk), blk = (int)(tile % nblk);
    const int k = ks.iters[r];
    if (accumulate && k == 0) continue;
    const long long g0 = (long long)blk * (CHUNK / W) + threadIdx.x;
    C<Tx>* xr = x + r * n;
    const double2* yr = ks.y + (long long)r * ks.m;
    C<Tx> acc[EPT];
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk)
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const long long e = (g0 + (long long)kk * NT) * W + u;
        acc[kk * W + u] = (accumulate && e < n) ? xr[e] : czero<Tx>();
      }
    for (int q0 = 0; q0 < k; q0 += G) {
      uint4 raw[G][VPT];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const SB* vr = V + (long long)(q0 + q) * vstride + r * rs;
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          const long long g = g0 + (long long)kk * NT;
          raw[q][kk] = (q0 + q < k && g * W < n) ? ldraw(vr, g) : make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const C<Tx> yi = (q0 + q < k) ? cvt_to<Tx>(yr[q0 + q]) : czero<Tx>();
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          static_for<W>([&](auto U) {
            const auto v = unpk<U.value>(raw[q][kk], (const SB*)nullptr);
            const Tx vx = (Tx)v.x, vy = (Tx)v.y;
            acc[kk * W + U.value].x += vx * yi.x - vy * yi.y;
            acc[kk * W + U.value].y += vx * yi.y + vy * yi.x;
          });
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk)
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const long long e = (g0 + (long long)kk * NT) * W + u;
        if (e < n) xr[e] = acc[kk * W + u];
      }
  }
}

// The same update one element at a time, for bases whose rows are not
// 16-byte aligned (row length not a multiple of 16 bytes).
template <class SB, class Tx>
__global__ void __launch_bounds__(NT)
k_update_el(const SB* __restrict__ V, long long vstride, long long rs, KState ks,
         C<Tx>* __restrict__ x, int accumulate, long long n, int nrhs, int nblk) {
  constexpr int TILE = 512;
  __shared__ C<Tx> ys[TILE];
  for (long long tile = blockIdx.x; tile < (long long)nrhs * nblk; tile += gridDim.x) {
  const int r = (int)(tile / nblk), blk = (int)(tile % nblk);
  const int k = ks.iters[r];
  if (accumulate && k == 0) continue;
  const long long base = (long long)blk * CHUNK + threadIdx.x;
  C<Tx>* xr = x + r * n;
  C<Tx> acc[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const long long e = base + q * NT;
    acc[q] = (accumulate && e < n) ? xr[e] : czero<Tx>();
  }
  for (int t0 = 0; t0 < k; t0 += TILE) {
    const int cnt = min(TILE, k - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += NT)
      ys[q] = cvt_to<Tx>(ks.y[(long long)r * ks.m + t0 + q]);
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      const SB* vr = V + (long long)(t0 + i) * vstride + r * rs;
      const C<Tx> yi = ys[i];
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const long long e = base + q * NT;
        if (e < n) {
          const C<Tx> v = ld2(vr, e);
          acc[q].x += (Tx)v.x * yi.x - (Tx)v.y * yi.y;
          acc[q].y += (Tx)v.x * yi.y + (Tx)v.y * yi.x;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const long long e = base + q * NT;
    if (e < n) xr[e] = acc[q];
  }
  }
}

// Kernels executed inside WHILE-node bodies (graph launches are counted on
// the host; the iterations of a device-side loop only here).
__device__ unsigned long long g_body_kernels_run;

// (a raised fault flag ends the loop too: a bounded wait ran out)
__global__ void k_loop_begin(const int* alldone, const int* fault, int* it,
                             cudaGraphConditionalHandle h) {
  *it = 0;
  cudaGraphSetConditional(h, (*alldone || (fault && *fault)) ? 0u : 1u);
}

__global__ void k_loop_next(const int* alldone, const int* fault, int* it, int maxit,
                            const int* body_kernels, cudaGraphConditionalHandle h) {
  const int k = *it + 1;
  *it = k;
  atomicAdd(&g_body_kernels_run, (unsigned long long)*body_kernels);
  cudaGraphSetConditional(h, (!*alldone && !(fault && *fault) && k < maxit) ? 1u : 0u);
}

// GCR step (Sec. 6.3's outer iteration): x += g u_k and r -= g c_k with
// g = hcol[r][0] = (c_k, r), and the partial ||r||^2 of the new residual.
__global__ void __launch_bounds__(NT)
k_gcr_update(double2* __restrict__ x, double2* __restrict__ res,
             const double2* __restrict__ u, const double2* __restrict__ c, long long n,
             KState ks) {
  __shared__ double red[NT / 32];
  const int r = blockIdx.y, blk = blockIdx.x;
  if (ks.done[r]) return;
  const double2 g = ks.hcol[(long long)r * (ks.m + 1)];
  double s = 0.0;
  for (int k = 0; k < EPT; ++k) {
    const long long e = (long long)blk * CHUNK + k * NT + threadIdx.x;
    if (e >= n) break;
    const long long id = r * n + e;
    const double2 uv = u[id], cv = c[id];
    double2 xv = x[id], rv = res[id];
    xv.x += g.x * uv.x - g.y * uv.y;
    xv.y += g.x * uv.y + g.y * uv.x;
    rv.x -= g.x * cv.x - g.y * cv.y;
    rv.y -= g.x * cv.y + g.y * cv.x;
    x[id] = xv;
    res[id] = rv;
    s += rv.x * rv.x + rv.y * rv.y;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) ks.npart[(long long)r * ks.nblk_max + blk] = t;
}

// GCR convergence after step k: ||r|| <= tol ||b|| (rnorm[r] = ||r||), a
// non-finite residual, or the cap; all-converged flag.
__global__ void k_gcr_check(KState ks, const double* __restrict__ rnorm, int nrhs,
                            double tol, int k, int maxit) {
  const int r = threadIdx.x;
  int d = 1;
  if (r < nrhs) {
    d = ks.done[r];
    if (!d) {
      const double res = rnorm[r];
      ks.iters[r] = k + 1;
      if (!isfinite(res)) {
        d = 1;
        ks.stat[r] = ST_NAN;
      } else if (res <= tol * ks.bnorm[r]) {
        d = 1;
      } else if (k + 1 >= maxit) {
        d = 1;
        ks.stat[r] = ST_NOT_CONVERGED;
      }
      ks.done[r] = d;
    }
  }
  const int all = __syncthreads_and(d);
  if (r == 0) *ks.alldone = all;
}

// Synthetic vectors for timing (values in [-1/2, 1/2) from an integer hash
// of the index); no result of the method depends on them.
template <class SB>
__global__ void k_tune_fill(SB* __restrict__ p, long long count, unsigned seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)e * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float a = (float)(h & 0xffffu) * (1.0f / 65536.0f) - 0.5f;
    const float b = (float)(h >> 16) * (1.0f / 65536.0f) - 0.5f;
    if constexpr (std::is_same<SB, double2>::value)
      p[e] = make_double2(a, b);
    else
      st2(p, e, make_float2(a, b));
  }
}
// Arnoldi state of a timing run: column j, every RHS below nrhs active.
__global__ void k_tune_state(KState ks, int nrhs, int j) {
  const int r = threadIdx.x;
  if (r == 0) *ks.jctr = j;
  if (r < nrhs) {
    ks.done[r] = 0;
    ks.reorth[r] = 0;
  }
}

__global__ void k_fill_int(int* p, int v, int count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) p[e] = v;
}
__global__ void k_copy_int(const int* s, int* d, int count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) d[e] = s[e];
}

}  // namespace

int krylov_nblk(long long n) { return (int)((n + CHUNK - 1) / CHUNK); }

namespace {
// Blocks of a persistent launch: at most as many as the GPU keeps resident
// (SMs x resident blocks per SM for this kernel), so the last wave is never
// a small fraction of the GPU; cached per kernel and device.
std::mutex g_grid_mu;
std::unordered_map<long long, int> g_grid_cap;

unsigned persistent_grid(const void* kern, long long tiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  const long long key = (long long)(uintptr_t)kern * 64 + dev;
  int cap = 0;
  {
    std::lock_guard<std::mutex> lock(g_grid_mu);
    auto it = g_grid_cap.find(key);
    if (it != g_grid_cap.end()) cap = it->second;
  }
  if (!cap) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, 0);
    cap = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    std::lock_guard<std::mutex> lock(g_grid_mu);
    g_grid_cap[key] = cap;
  }
  return (unsigned)(tiles < cap ? tiles : cap);
}
}  // namespace

namespace {
int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  cache[dev] = sms;
  return sms;
}
// opt a kernel in to the stage ring's dynamic shared memory (once per kernel)
void allow_stages(const void* kern) {
  static std::mutex mu;
  static std::unordered_map<const void*, bool> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done[kern]) return;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, RING_BYTES);
  done[kern] = true;
}
}  // namespace

template <class T, class SB>
void launch_mdot(const SB* V, long long vstride, long long rs, const C<T>* w,
                 long long n, int nrhs, const KState& ks, int pass, cudaStream_t st) {
  HZ_COUNT();
  const int nblk = krylov_nblk(n);
  if (ks.dotk == 1 || ks.dotk == 2) {
    const void* kern = ks.dotk == 1 ? (const void*)k_mdot_tma<T, SB, 8>
                                   : (const void*)k_mdot_tma<T, SB, 16>;
    allow_stages(kern);
    if (ks.dotk == 1)
      k_mdot_tma<T, SB, 8><<<sm_count(), 288, RING_BYTES, st>>>(V, vstride, rs, w, n, ks,
                                                               pass, nrhs, nblk);
    else
      k_mdot_tma<T, SB, 16><<<sm_count(), 544, RING_BYTES, st>>>(V, vstride, rs, w, n, ks,
                                                                pass, nrhs, nblk);
    return;
  }
  const unsigned grid = persistent_grid((const void*)k_mdot<T, SB>, (long long)nblk * nrhs);
  k_mdot<T, SB><<<grid, NT, 0, st>>>(V, vstride, rs, w, n, ks, pass, nrhs, nblk);
}
template <class T, class SB>
void launch_mdot_group(const GroupDesc& gd, int pass, cudaStream_t st) {
  HZ_COUNT();
  const unsigned grid =
      persistent_grid((const void*)k_mdot_group<T, SB>, gd.start[gd.count]);
  k_mdot_group<T, SB><<<grid, NT, 0, st>>>(gd, pass);
}
template <class T, class SB>
void launch_maxpy_group(const GroupDesc& gd, int pass, cudaStream_t st) {
  HZ_COUNT();
  const unsigned grid =
      persistent_grid((const void*)k_maxpy_group<T, SB>, gd.start[gd.count]);
  k_maxpy_group<T, SB><<<grid, NT, 0, st>>>(gd, pass);
}
void launch_reduce_cols(const KState& ks, long long n, int nrhs, int pass,
                        cudaStream_t st) {
  HZ_COUNT();
  const int wpb = NT / 32;
  k_reduce_cols<<<dim3((ks.m + 1 + wpb - 1) / wpb, nrhs), NT, 0, st>>>(
      ks, krylov_nblk(n), pass);
}
template <class T, class SB>
void launch_maxpy(const SB* V, long long vstride, long long rs, C<T>* w,
                  long long n, int nrhs, const KState& ks, int pass, cudaStream_t st) {
  HZ_COUNT();
  const int nblk = krylov_nblk(n);
  if (ks.updk == 1 || ks.updk == 2) {
    const void* kern = ks.updk == 1 ? (const void*)k_maxpy_tma<T, SB, 8>
                                   : (const void*)k_maxpy_tma<T, SB, 16>;
    allow_stages(kern);
    const long long tiles = (long long)nblk * nrhs;
    const unsigned grid = (unsigned)(tiles < sm_count() ? tiles : sm_count());
    if (ks.updk == 1)
      k_maxpy_tma<T, SB, 8><<<grid, 288, RING_BYTES, st>>>(V, vstride, rs, w, n, ks, pass,
                                                          nrhs, nblk);
    else
      k_maxpy_tma<T, SB, 16><<<grid, 544, RING_BYTES, st>>>(V, vstride, rs, w, n, ks, pass,
                                                           nrhs, nblk);
    return;
  }
  const unsigned grid = persistent_grid((const void*)k_maxpy<T, SB>, (long long)nblk * nrhs);
  k_maxpy<T, SB><<<grid, NT, 0, st>>>(V, vstride, rs, w, n, ks, pass, nrhs, nblk);
}
void launch_reorth_decide(const KState& ks, long long n, int nrhs, double eta,
                          cudaStream_t st) {
  HZ_COUNT();
  k_reorth_decide<<<nrhs, NT, 0, st>>>(ks, krylov_nblk(n), eta);
}
template <class T>
void launch_norm2_part(VRef<T> w, long long n, int nrhs, const KState& ks,
                       const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_norm2_part<T><<<dim3(krylov_nblk(n), nrhs), NT, 0, st>>>(w, n, ks, done);
}
void launch_reduce_norm(const KState& ks, long long n, int nrhs, double* out,
                        int sqrt_it, cudaStream_t st) {
  HZ_COUNT();
  k_reduce_norm<<<nrhs, NT, 0, st>>>(ks, krylov_nblk(n), out, sqrt_it);
}
void launch_krylov_init(const KState& ks, int nrhs, const int* done_in,
                        const double* bnorm_src, double tol, cudaStream_t st) {
  HZ_COUNT();
  k_krylov_init<<<1, 1024, 0, st>>>(ks, nrhs, done_in, bnorm_src, tol);
}
template <class T, class SB>
void launch_scale_into(VRef<T> w, VRefE<SB> out, long long rs, const double* s,
                       long long n, int nrhs, const int* done, cudaStream_t st,
                       C<T>* copy) {
  HZ_COUNT();
  long long nb = (rs + 1023) / 1024;
  if (nb > 1024) nb = 1024;
  k_scale_into<T, SB><<<dim3((unsigned)nb, nrhs), 256, 0, st>>>(w, out, rs, s, n, done,
                                                                copy);
}
void launch_givens(const KState& ks, int nrhs, double tol, int maxit,
                   cudaStream_t st) {
  HZ_COUNT();
  const size_t smem = (size_t)(ks.m + 2) * sizeof(double2) +
                      (size_t)ks.m * (sizeof(double2) + sizeof(double));
  static std::once_flag once;
  std::call_once(once, [] {
    // the largest basis (3000 columns) needs 120 KB
    cudaFuncSetAttribute((const void*)k_givens, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(3002 * sizeof(double2) + 3000 * (sizeof(double2) + sizeof(double))));
  });
  k_givens<<<nrhs, 128, smem, st>>>(ks, tol, maxit);
  HZ_COUNT();
  k_givens_finish<<<1, 1024, 0, st>>>(ks, nrhs);
}
void launch_trisolve(const KState& ks, int nrhs, cudaStream_t st) {
  HZ_COUNT();
  k_trisolve<<<nrhs, 128, (size_t)ks.m * sizeof(double2), st>>>(ks);
}
template <class SB, class Tx>
void launch_update(const SB* V, long long vstride, long long rs, const KState& ks,
                   C<Tx>* x, int accumulate, long long n, int nrhs,
                   cudaStream_t st) {
  HZ_COUNT();
  const int nblk = krylov_nblk(n);
  // the 16-byte group loads need every row 16-byte aligned
  const bool aligned = reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
                       (rs * (long long)sizeof(SB)) % 16 == 0 &&
                       (vstride * (long long)sizeof(SB)) % 16 == 0;
  if (!aligned) {
    const unsigned grid =
        persistent_grid((const void*)k_update_el<SB, Tx>, (long long)nblk * nrhs);
    k_update_el<SB, Tx><<<grid, NT, 0, st>>>(V, vstride, rs, ks, x, accumulate, n, nrhs, nblk);
    return;
  }
  const unsigned grid = persistent_grid((const void*)k_update<SB, Tx>, (long long)nblk * nrhs);
  k_update<SB, Tx><<<grid, NT, 0, st>>>(V, vstride, rs, ks, x, accumulate, n, nrhs, nblk);
}
void launch_fill_int(int* p, int v, int count, cudaStream_t st) {
  HZ_COUNT();
  k_fill_int<<<(count + 255) / 256, 256, 0, st>>>(p, v, count);
}
void launch_gcr_update(double2* x, double2* r, const double2* u, const double2* c,
                       long long n, int nrhs, const KState& ks, cudaStream_t st) {
  HZ_COUNT();
  k_gcr_update<<<dim3(krylov_nblk(n), nrhs), NT, 0, st>>>(x, r, u, c, n, ks);
}
void launch_gcr_check(const KState& ks, const double* rnorm, int nrhs, double tol, int k,
                      int maxit, cudaStream_t st) {
  HZ_COUNT();
  k_gcr_check<<<1, 1024, 0, st>>>(ks, rnorm, nrhs, tol, k, maxit);
}
template <class SB>
void launch_tune_fill(SB* p, long long count, unsigned seed, cudaStream_t st) {
  HZ_COUNT();
  long long nb = (count + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_tune_fill<SB><<<(unsigned)nb, 256, 0, st>>>(p, count, seed);
}
template void launch_tune_fill<double2>(double2*, long long, unsigned, cudaStream_t);
template void launch_tune_fill<float2>(float2*, long long, unsigned, cudaStream_t);
template void launch_tune_fill<__half2>(__half2*, long long, unsigned, cudaStream_t);
void launch_tune_state(const KState& ks, int nrhs, int j, cudaStream_t st) {
  HZ_COUNT();
  k_tune_state<<<1, 1024, 0, st>>>(ks, nrhs, j);
}
void launch_loop_begin(const int* alldone, const int* fault, int* it,
                       cudaGraphConditionalHandle h, cudaStream_t st) {
  HZ_COUNT();
  k_loop_begin<<<1, 1, 0, st>>>(alldone, fault, it, h);
}
void launch_loop_next(const int* alldone, const int* fault, int* it, int maxit,
                      const int* body_kernels, cudaGraphConditionalHandle h,
                      cudaStream_t st) {
  HZ_COUNT();
  k_loop_next<<<1, 1, 0, st>>>(alldone, fault, it, maxit, body_kernels, h);
}
namespace {
__global__ void k_all_of(FlagSet fs, int* out) {
  int a = 1;
  for (int i = 0; i < fs.n; ++i) a &= (*fs.f[i] != 0) ? 1 : 0;
  *out = a;
}
}  // namespace
void launch_all_of(const FlagSet& fs, int* out, cudaStream_t st) {
  HZ_COUNT();
  k_all_of<<<1, 1, 0, st>>>(fs, out);
}

unsigned long long graph_body_kernels_run() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_body_kernels_run, sizeof v) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}
void launch_copy_int(const int* src, int* dst, int count, cudaStream_t st) {
  HZ_COUNT();
  k_copy_int<<<(count + 255) / 256, 256, 0, st>>>(src, dst, count);
}

#define HZ_KINST(T, SB)                                                         \
  template void launch_mdot<T, SB>(const SB*, long long, long long, const C<T>*, \
                                   long long, int, const KState&, int,          \
                                   cudaStream_t);                               \
  template void launch_maxpy<T, SB>(const SB*, long long, long long, C<T>*,      \
                                    long long, int, const KState&, int,         \
                                    cudaStream_t);                              \
  template void launch_scale_into<T, SB>(VRef<T>, VRefE<SB>, long long,         \
                                         const double*, long long, int,         \
                                         const int*, cudaStream_t, C<T>*);      \
  template void launch_update<SB, T>(const SB*, long long, long long,           \
                                     const KState&, C<T>*, int, long long, int, \
                                     cudaStream_t);                             \
  template void launch_mdot_group<T, SB>(const GroupDesc&, int, cudaStream_t);  \
  template void launch_maxpy_group<T, SB>(const GroupDesc&, int, cudaStream_t);

template void launch_norm2_part<double>(VRef<double>, long long, int, const KState&,
                                        const int*, cudaStream_t);
template void launch_norm2_part<float>(VRef<float>, long long, int, const KState&,
                                       const int*, cudaStream_t);

HZ_KINST(double, double2)
HZ_KINST(float, float2)
HZ_KINST(float, __half2)

}  // namespace hz
