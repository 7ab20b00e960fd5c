// Field-split additive Schwarz kernels (Sec. 3.2: AS1 / AS2 Vanka blocks
// solved by LU, Jacobi on the lumped mass K_u^s) and the coarse direct solve.
//
// Set-up: every block A_jj = A_l[I_j, I_j] is gathered from the float64 CSR
// straight into shared memory and inverted in place by unpivoted
// Gauss-Jordan elimination in float64.  The unknown order inside a block is
// the J2 order, which puts displacement/velocity before pressure, so the
// leading pivots are those of the (positive definite) momentum / ALE blocks
// and the pressure pivots are Schur complements.  Blocks larger than one
// CTA's shared memory are split by rows over a thread-block cluster of 2-8
// CTAs; the pivot row of each step is read by the other CTAs through
// distributed shared memory.  The inverse is stored row-major (rows padded
// to 16 bytes) in float64 or float32.
//
// Apply (the per-iteration hot loop): y = A_jj^{-1} r_j is a dense GEMV that
// streams each stored inverse once from HBM with 16-byte vector loads; the
// blocks overlap, so each block row's result goes to its own slot of a
// staging vector (one slot per entry of the block index lists), and a second
// kernel combines them owner by owner: dof i adds W_i times its slots in
// block order, the additive formula's sum over j in a fixed order, so the
// smoother is bitwise repeatable.  Passes of the multiplicative sweep hold
// non-overlapping blocks and add into the correction directly.  Jacobi rows
// (u^s and fixed dofs) ride in the apply launch as their own work items.
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "context.h"

namespace cg = cooperative_groups;

namespace fsi {

namespace {

constexpr int GJ_THREADS = 256;

struct GJParams {
    const int32_t *blk_ptr, *blk_idx;
    const int64_t *blk_off;
    const int32_t *row_ptr, *col;
    const double *val;
    void *inv;                 // double, float or __half
    float *scale;              // float16 storage: per block row
    int storage;               // 0 float64, 1 float32, 2 float16 + row scale
    int rows_per_cta;          // R
    int *flags;
};

__device__ __forceinline__ int find_local(const int32_t *idx, int n, int c) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = idx[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid;
    }
    return -1;
}

template <int C>
__global__ void __launch_bounds__(GJ_THREADS) block_gj_kernel(GJParams P) {
    extern __shared__ double sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (C > 1) ? (int)cluster.block_rank() : 0;
    const int blk = blockIdx.x / C;
    const int s0 = P.blk_ptr[blk];
    const int n = P.blk_ptr[blk + 1] - s0;
    const int32_t *idx = P.blk_idx + s0;
    const int R = P.rows_per_cta;
    const int ld = R > 0 ? n : 0;
    const int r0 = rank * R;
    const int nr = max(0, min(R, n - r0));        // rows held by this CTA
    double *A = sm;                               // [R][n]
    double *prow = sm + (size_t)R * n;            // [2][n] pivot rows published to the cluster
    double *pl = prow + 2 * (size_t)n;            // [n] local copy of the pivot row
    double *fc = pl + n;                          // [R] column k of the local rows
    // gather the local rows from the CSR
    for (int t = threadIdx.x; t < nr * n; t += blockDim.x) A[t] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
    for (int li = warp; li < nr; li += nwarps) {
        const int g = idx[r0 + li];
        for (int k = P.row_ptr[g] + lane; k < P.row_ptr[g + 1]; k += 32) {
            const int pos = find_local(idx, n, P.col[k]);
            if (pos >= 0) A[(size_t)li * ld + pos] = P.val[k];
        }
    }
    __syncthreads();
    if (C > 1) cluster.sync();
    bool bad = false;
    for (int k = 0; k < n; ++k) {
        const int owner = k / R;
        const int buf = k & 1;
        if (rank == owner) {
            const int li = k - r0;
            double piv = A[(size_t)li * ld + k];
            if (!(fabs(piv) > 1e-300) || !isfinite(piv)) {
                bad = true;
                piv = 1.0;
            }
            const double ip = 1.0 / piv;
            for (int j = threadIdx.x; j < n; j += blockDim.x)
                prow[buf * n + j] = (j == k) ? ip : A[(size_t)li * ld + j] * ip;
        }
        if (C > 1) cluster.sync(); else __syncthreads();
        const double *src = prow + buf * n;
        if (C > 1) src = cluster.map_shared_rank(prow + buf * n, owner);
        for (int j = threadIdx.x; j < n; j += blockDim.x) pl[j] = src[j];
        for (int li = threadIdx.x; li < nr; li += blockDim.x) fc[li] = A[(size_t)li * ld + k];
        __syncthreads();
        const double ip = pl[k];
        for (int t = threadIdx.x; t < nr * n; t += blockDim.x) {
            const int li = t / n, j = t - li * n;
            const int i = r0 + li;
            double v;
            if (i == k) v = pl[j];
            else if (j == k) v = -fc[li] * ip;
            else v = A[t] - fc[li] * pl[j];
            A[t] = v;
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicExch(P.flags, 1);
    // keep peers' shared memory alive until every CTA stopped reading it
    if (C > 1) cluster.sync();
    const int64_t off = P.blk_off[blk];
    if (P.storage == 2) {
        // row-normalised float16: scale = max |row|, entries in [-1, 1]
        const int ldo = (n + 7) & ~7;
        __half *out = static_cast<__half *>(P.inv) + off;
        const int warp2 = threadIdx.x / 32, lane2 = threadIdx.x % 32;
        for (int li = warp2; li < nr; li += blockDim.x / 32) {
            double m = 0.0;
            for (int j = lane2; j < n; j += 32) m = fmax(m, fabs(A[(size_t)li * ld + j]));
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            const double sc = m > 0.0 ? m : 1.0;
            if (lane2 == 0) P.scale[s0 + r0 + li] = (float)sc;
            const double isc = 1.0 / sc;
            for (int j = lane2; j < ldo; j += 32)
                out[(size_t)(r0 + li) * ldo + j] = __float2half_rn(j < n ? (float)(A[(size_t)li * ld + j] * isc) : 0.0f);
        }
    } else if (P.storage == 1) {
        const int ldo = (n + 3) & ~3;
        float *out = static_cast<float *>(P.inv) + off;
        for (int t = threadIdx.x; t < nr * ldo; t += blockDim.x) {
            const int li = t / ldo, j = t - li * ldo;
            out[(size_t)(r0 + li) * ldo + j] = (j < n) ? (float)A[(size_t)li * ld + j] : 0.0f;
        }
    } else {
        const int ldo = (n + 1) & ~1;
        double *out = static_cast<double *>(P.inv) + off;
        for (int t = threadIdx.x; t < nr * ldo; t += blockDim.x) {
            const int li = t / ldo, j = t - li * ldo;
            out[(size_t)(r0 + li) * ldo + j] = (j < n) ? A[(size_t)li * ld + j] : 0.0;
        }
    }
}

// vector types for the GEMV stream
template <class T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int w = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int w = 2; };

__device__ __forceinline__ float dotv(const float4 &a, const float4 &b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double dotv(const double2 &a, const double2 &b) {
    return a.x * b.x + a.y * b.y;
}

template <class T>
__device__ __forceinline__ typename Vec<T>::type ld_stream(const typename Vec<T>::type *p) {
    return __ldcs(p);   // streaming: read once, evict first
}

// Sum 4 per-lane row partials over the warp with 6 shuffles (a transposing
// butterfly): afterwards lane 8 q holds the total of row q (q = 0..3).
template <class T>
__device__ __forceinline__ T warp_reduce4(const T (&a)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    const T s0 = b4 ? a[0] : a[2], s1 = b4 ? a[1] : a[3];
    const T k0 = (b4 ? a[2] : a[0]) + __shfl_xor_sync(0xffffffffu, s0, 16);
    const T k1 = (b4 ? a[3] : a[1]) + __shfl_xor_sync(0xffffffffu, s1, 16);
    T v = (b3 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

constexpr int APPLY_THREADS = 128;
constexpr int MAX_BLOCK = 1024;
constexpr int RPW = 4;          // rows per warp iteration (independent 16-byte loads in flight)

// One work item = rows [r0, r1) of block j (whole blocks on large levels,
// row chunks on small levels so that every SM has work).
template <class T>
__global__ void __launch_bounds__(APPLY_THREADS) block_apply_kernel(const int4 *__restrict__ items,
                                                                    const int32_t *__restrict__ blk_ptr,
                                                                    const int32_t *__restrict__ blk_idx,
                                                                    const int64_t *__restrict__ blk_off,
                                                                    const T *__restrict__ blk_w,
                                                                    const T *__restrict__ inv,
                                                                    const int32_t *__restrict__ jac_idx,
                                                                    const T *__restrict__ jac_inv,
                                                                    const T *__restrict__ r, T *__restrict__ x,
                                                                    T omega, T *__restrict__ stage) {
    using V = typename Vec<T>::type;
    constexpr int VW = Vec<T>::w;
    __shared__ __align__(16) T rs[MAX_BLOCK];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, r0 = it.y, r1 = it.z;
    pdl_wait();
    if (blk < 0) {               // Jacobi rows [r0, r1) of the jac list (u^s and fixed dofs)
        for (int k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int ld = (n + VW - 1) / VW * VW;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) rs[i] = (i < n) ? r[blk_idx[s0 + i]] : T(0);
    __syncthreads();
    const V *M = reinterpret_cast<const V *>(inv + blk_off[blk]);
    const V *rv = reinterpret_cast<const V *>(rs);
    const int nv = ld / VW;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int NW = APPLY_THREADS / 32;
    for (int i = r0 + warp * RPW; i < r1; i += NW * RPW) {
        T a[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) a[q] = 0;
        for (int c = lane; c < nv; c += 32) {
            const V rc = rv[c];
            V m[RPW];
#pragma unroll
            for (int q = 0; q < RPW; ++q)
                if (i + q < r1) m[q] = ld_stream<T>(M + (size_t)(i + q) * nv + c);
#pragma unroll
            for (int q = 0; q < RPW; ++q)
                if (i + q < r1) a[q] += dotv(m[q], rc);
        }
        const T v = warp_reduce4<T>(a, lane);
        const int q = lane >> 3;
        if ((lane & 7) == 0 && i + q < r1) {
            const int g = s0 + i + q;
            if (stage) stage[g] = v;
            else atomicAdd(&x[blk_idx[g]], omega * blk_w[g] * v);
        }
    }
}

// transposed apply: y = A_jj^{-T} (W_j r_j); columns [r0, r1) of the item,
// thread per column, rows streamed
template <class T>
__global__ void __launch_bounds__(APPLY_THREADS) block_apply_t_kernel(const int4 *__restrict__ items,
                                                                      const int32_t *__restrict__ blk_ptr,
                                                                      const int32_t *__restrict__ blk_idx,
                                                                      const int64_t *__restrict__ blk_off,
                                                                      const T *__restrict__ blk_w,
                                                                      const T *__restrict__ inv,
                                                                      const int32_t *__restrict__ jac_idx,
                                                                      const T *__restrict__ jac_inv,
                                                                      const T *__restrict__ r, T *__restrict__ x,
                                                                      T omega, T *__restrict__ stage) {
    constexpr int VW = Vec<T>::w;
    __shared__ T rs[MAX_BLOCK];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, c0 = it.y, c1 = it.z;
    pdl_wait();
    if (blk < 0) {               // Jacobi rows: diagonal, its own transpose
        for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int ld = (n + VW - 1) / VW * VW;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = blk_w[s0 + i] * r[blk_idx[s0 + i]];
    __syncthreads();
    const T *M = inv + blk_off[blk];
    for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        T acc = 0;
        for (int i = 0; i < n; ++i) acc += M[(size_t)i * ld + j] * rs[i];
        if (stage) stage[s0 + j] = acc;
        else atomicAdd(&x[blk_idx[s0 + j]], omega * acc);
    }
}

// float16 storage (row-normalised, float32 scale per row), float32 vectors
__device__ __forceinline__ float dot8(const uint4 &m, const float4 &a, const float4 &b) {
    const __half2 *h = reinterpret_cast<const __half2 *>(&m);
    const float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
    const float2 f2 = __half22float2(h[2]), f3 = __half22float2(h[3]);
    return f0.x * a.x + f0.y * a.y + f1.x * a.z + f1.y * a.w + f2.x * b.x + f2.y * b.y + f3.x * b.z + f3.y * b.w;
}

template <int HR>
__global__ void __launch_bounds__(APPLY_THREADS) block_apply_h_kernel(const int4 *__restrict__ items,
                                                                      const int32_t *__restrict__ blk_ptr,
                                                                      const int32_t *__restrict__ blk_idx,
                                                                      const int64_t *__restrict__ blk_off,
                                                                      const float *__restrict__ blk_w,
                                                                      const __half *__restrict__ inv,
                                                                      const float *__restrict__ scale,
                                                                      const int32_t *__restrict__ jac_idx,
                                                                      const float *__restrict__ jac_inv,
                                                                      const float *__restrict__ r, float *__restrict__ x,
                                                                      float omega, float *__restrict__ stage) {
    __shared__ __align__(16) float rs[MAX_BLOCK];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, r0 = it.y, r1 = it.z;
    pdl_wait();
    if (blk < 0) {
        for (int k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int ld = (n + 7) & ~7;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) rs[i] = (i < n) ? r[blk_idx[s0 + i]] : 0.0f;
    __syncthreads();
    const uint4 *M = reinterpret_cast<const uint4 *>(inv + blk_off[blk]);
    const float4 *rv = reinterpret_cast<const float4 *>(rs);
    const int nv = ld / 8;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int NW = APPLY_THREADS / 32;
    for (int i = r0 + warp * HR; i < r1; i += NW * HR) {
        float a[HR];
#pragma unroll
        for (int q = 0; q < HR; ++q) a[q] = 0.0f;
        for (int c = lane; c < nv; c += 32) {
            const float4 ra = rv[2 * c], rb = rv[2 * c + 1];
            uint4 m[HR];
#pragma unroll
            for (int q = 0; q < HR; ++q)
                if (i + q < r1) m[q] = __ldcs(M + (size_t)(i + q) * nv + c);
#pragma unroll
            for (int q = 0; q < HR; ++q)
                if (i + q < r1) a[q] += dot8(m[q], ra, rb);
        }
        static_assert(HR == 4, "the transposing reduction sums 4 rows");
        const float v = warp_reduce4<float>(a, lane);
        const int q = lane >> 3;
        if ((lane & 7) == 0 && i + q < r1) {
            const int g = s0 + i + q;
            if (stage) stage[g] = scale[g] * v;
            else atomicAdd(&x[blk_idx[g]], omega * blk_w[g] * scale[g] * v);
        }
    }
}

// Blocks of at most 256 dofs (every 2D block): each lane owns one 16-byte
// chunk of a row, so the loads of a 4-row group are one uint4 per lane and
// row.  The first group's loads are issued before the residual gather (the
// HBM and L2 latencies overlap) and the next group's loads are in flight
// while the current group is reduced and scattered.
__global__ void __launch_bounds__(APPLY_THREADS, 12) block_apply_h_pipe_kernel(const int4 *__restrict__ items,
                                                                           const int32_t *__restrict__ blk_ptr,
                                                                           const int32_t *__restrict__ blk_idx,
                                                                           const int64_t *__restrict__ blk_off,
                                                                           const float *__restrict__ blk_w,
                                                                           const __half *__restrict__ inv,
                                                                           const float *__restrict__ scale,
                                                                           const int32_t *__restrict__ jac_idx,
                                                                           const float *__restrict__ jac_inv,
                                                                           const float *__restrict__ r,
                                                                           float *__restrict__ x, float omega,
                                                                           float *__restrict__ stage) {
    __shared__ __align__(16) float rs[256];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, r0 = it.y, r1 = it.z;
    if (blk < 0) {
        pdl_wait();
        for (int k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int ld = (n + 7) & ~7;
    const int nv = ld / 8;                      // <= 32
    const uint4 *M = reinterpret_cast<const uint4 *>(inv + blk_off[blk]);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int NW = APPLY_THREADS / 32;
    const bool col_ok = lane < nv;
    int i = r0 + warp * 4;
    uint4 m[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        m[q] = (col_ok && i + q < r1) ? __ldcs(M + (size_t)(i + q) * nv + lane) : make_uint4(0, 0, 0, 0);
    pdl_wait();                                 // the inverse rows above are static; r is not
    for (int k = threadIdx.x; k < ld; k += blockDim.x) rs[k] = (k < n) ? r[blk_idx[s0 + k]] : 0.0f;
    __syncthreads();
    const float4 *rv = reinterpret_cast<const float4 *>(rs);
    const float4 ra = col_ok ? rv[2 * lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 rb = col_ok ? rv[2 * lane + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (; i < r1; i += NW * 4) {
        const int in = i + NW * 4;
        uint4 mn[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mn[q] = (col_ok && in + q < r1) ? __ldcs(M + (size_t)(in + q) * nv + lane) : make_uint4(0, 0, 0, 0);
        float a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = dot8(m[q], ra, rb);
        const float v = warp_reduce4<float>(a, lane);
        const int q = lane >> 3;
        if ((lane & 7) == 0 && i + q < r1) {
            const int g = s0 + i + q;
            if (stage) stage[g] = scale[g] * v;
            else atomicAdd(&x[blk_idx[g]], omega * blk_w[g] * scale[g] * v);
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) m[qq] = mn[qq];
    }
}

// transposed: A^{-1} = D_s M (D_s row scales), so A^{-T} W r = M^T (D_s W r)
// Transposed float16 apply for blocks of at most 256 dofs, streamed by rows
// like the forward apply: y[c] = sum_i M[i][c] (scale_i w_i r_i) for the
// item's columns [c0, c1).  Lane q of a warp owns the 16-byte chunk q of the
// item's columns in every row it visits; the warps take every fourth row
// (4 rows in flight per lane) and their column partials meet in shared
// memory before the scatter-add.  Replaces one thread per column walking all
// rows (171 dependent 2-byte loads per thread).
__global__ void __launch_bounds__(APPLY_THREADS) block_apply_h_tr_kernel(const int4 *__restrict__ items,
                                                                         const int32_t *__restrict__ blk_ptr,
                                                                         const int32_t *__restrict__ blk_idx,
                                                                         const int64_t *__restrict__ blk_off,
                                                                         const float *__restrict__ blk_w,
                                                                         const __half *__restrict__ inv,
                                                                         const float *__restrict__ scale,
                                                                         const int32_t *__restrict__ jac_idx,
                                                                         const float *__restrict__ jac_inv,
                                                                         const float *__restrict__ r,
                                                                         float *__restrict__ x, float omega,
                                                                         float *__restrict__ stage) {
    constexpr int NW = APPLY_THREADS / 32;
    __shared__ float rs[256];
    __shared__ float part[NW][256];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, c0 = it.y, c1 = it.z;
    pdl_wait();
    if (blk < 0) {
        for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int nv = ((n + 7) & ~7) / 8;            // 16-byte chunks per stored row
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = scale[s0 + i] * blk_w[s0 + i] * r[blk_idx[s0 + i]];
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int k0 = c0 / 8;                          // c0 is a multiple of 16
    const int kk = k0 + lane;
    const bool ok = kk < nv && lane * 8 < c1 - c0;     // chunk meets the item's columns
    const uint4 *M = reinterpret_cast<const uint4 *>(inv + blk_off[blk]);
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
    for (int i = warp; i < n; i += 4 * NW) {
        uint4 m[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = i + q * NW;
            m[q] = (ok && row < n) ? __ldcs(M + (size_t)row * nv + kk) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = i + q * NW;
            const float v = row < n ? rs[row] : 0.f;
            const __half2 *h = reinterpret_cast<const __half2 *>(&m[q]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __half22float2(h[e]);
                acc[2 * e] += f.x * v;
                acc[2 * e + 1] += f.y * v;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) part[warp][lane * 8 + e] = acc[e];
    __syncthreads();
    for (int c = threadIdx.x; c < c1 - c0; c += blockDim.x) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += part[w][c];
        if (stage) stage[s0 + c0 + c] = sum;
        else atomicAdd(&x[blk_idx[s0 + c0 + c]], omega * sum);
    }
}

__global__ void __launch_bounds__(APPLY_THREADS) block_apply_h_t_kernel(const int4 *__restrict__ items,
                                                                        const int32_t *__restrict__ blk_ptr,
                                                                        const int32_t *__restrict__ blk_idx,
                                                                        const int64_t *__restrict__ blk_off,
                                                                        const float *__restrict__ blk_w,
                                                                        const __half *__restrict__ inv,
                                                                        const float *__restrict__ scale,
                                                                        const int32_t *__restrict__ jac_idx,
                                                                        const float *__restrict__ jac_inv,
                                                                        const float *__restrict__ r, float *__restrict__ x,
                                                                        float omega, float *__restrict__ stage) {
    __shared__ float rs[MAX_BLOCK];
    pdl_trigger();
    const int4 it = items[blockIdx.x];
    const int blk = it.x, c0 = it.y, c1 = it.z;
    pdl_wait();
    if (blk < 0) {
        for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
            const int i = jac_idx[k];
            x[i] += omega * r[i] * jac_inv[k];
        }
        return;
    }
    const int s0 = blk_ptr[blk];
    const int n = blk_ptr[blk + 1] - s0;
    const int ld = (n + 7) & ~7;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = scale[s0 + i] * blk_w[s0 + i] * r[blk_idx[s0 + i]];
    __syncthreads();
    const __half *M = inv + blk_off[blk];
    for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        float acc = 0.0f;
        for (int i = 0; i < n; ++i) acc += __half2float(M[(size_t)i * ld + j]) * rs[i];
        if (stage) stage[s0 + j] = acc;
        else atomicAdd(&x[blk_idx[s0 + j]], omega * acc);
    }
}

// Owner-computes combination of the staged block results (additive Schwarz,
// Sec. 3.2): owner d (a dof covered by at least one block) sums
// w_d * stage[k] over its slots k in block order and adds omega times the sum
// to x.  Forward apply: w_d = 1 / multiplicity (the weights W_j); transposed
// apply: the weights were applied to r before the block products, w = 1.
template <class T>
__global__ void __launch_bounds__(256) block_gather_kernel(const int32_t *__restrict__ own_dof,
                                                         const int32_t *__restrict__ own_ptr,
                                                         const int32_t *__restrict__ own_pos,
                                                         const T *__restrict__ own_w, int64_t m,
                                                         const T *__restrict__ stage, T *__restrict__ x,
                                                         T omega, int weighted) {
    pdl_trigger();
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= m) { pdl_wait(); return; }
    const int k0 = own_ptr[d], k1 = own_ptr[d + 1], i = own_dof[d];
    const T w = weighted ? own_w[d] : T(1);
    pdl_wait();
    T acc = 0;
    for (int k = k0; k < k1; ++k) acc += w * stage[own_pos[k]];
    x[i] += omega * acc;
}

template <class T>
__global__ void jacobi_kernel(const int32_t *__restrict__ idx, const T *__restrict__ dinv, int64_t n,
                              const T *__restrict__ r, T *__restrict__ x, T omega) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = idx[k];
        x[i] += omega * r[i] * dinv[k];
    }
}

// ---- coarse level: Gauss-Jordan with partial pivoting on [A | I] ----
__global__ void coarse_pivot_kernel(double *M, int64_t n, int64_t k, int *flags) {
    // one CTA: argmax |M[i][k]|, i >= k; swap rows; scale row k
    __shared__ double best[1024];
    __shared__ int64_t bidx[1024];
    const int64_t w = 2 * n;
    double bv = -1.0;
    int64_t bi = k;
    for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
        const double v = fabs(M[i * w + k]);
        if (v > bv) { bv = v; bi = i; }
    }
    best[threadIdx.x] = bv;
    bidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = best[threadIdx.x + s];
            const int64_t oi = bidx[threadIdx.x + s];
            if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
                best[threadIdx.x] = o;
                bidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    __shared__ double spv;
    const int64_t p = bidx[0];
    if (threadIdx.x == 0) spv = M[p * w + k];
    __syncthreads();                       // every thread has p and the pivot before any swap
    const double pv = spv;
    if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
        if (threadIdx.x == 0) atomicExch(flags, 1);
        return;
    }
    const double ip = 1.0 / pv;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) {
        const double a = M[k * w + j], b = M[p * w + j];
        M[p * w + j] = a;
        M[k * w + j] = b * ip;
    }
}

__global__ void coarse_elim_kernel(double *M, int64_t n, int64_t k) {
    const int64_t w = 2 * n;
    const int64_t i = blockIdx.x;
    if (i == k) return;
    const double f = M[i * w + k];
    __syncthreads();
    if (f == 0.0) return;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[i * w + j] -= f * M[k * w + j];
}

__global__ void coarse_init_kernel(const int32_t *ptr, const int32_t *col, const double *val, int64_t n, double *M) {
    const int64_t w = 2 * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * w; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / w, j = t % w;
        M[t] = (j == n + i) ? 1.0 : 0.0;
    }
}
__global__ void coarse_fill_kernel(const int32_t *ptr, const int32_t *col, const double *val, int64_t n, double *M) {
    const int64_t w = 2 * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) M[i * w + col[k]] = val[k];
}
__global__ void coarse_extract_kernel(const double *M, int64_t n, double *inv) {
    const int64_t w = 2 * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, j = t % n;
        inv[t] = M[i * w + n + j];
    }
}

template <class T>
__global__ void dense_gemv_kernel(const double *__restrict__ M, int64_t n, const T *__restrict__ x, T *__restrict__ y) {
    pdl_trigger();
    pdl_wait();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    const int nwarps = gridDim.x * blockDim.x / 32;
    for (int64_t i = warp; i < n; i += nwarps) {
        double acc = 0.0;
        for (int64_t j = lane; j < n; j += 32) acc += M[i * n + j] * (double)x[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[i] = (T)acc;
    }
}
template <class T>
__global__ void dense_gemv_t_kernel(const double *__restrict__ M, int64_t n, const T *__restrict__ x, T *__restrict__ y) {
    pdl_trigger();
    pdl_wait();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) acc += M[i * n + j] * (double)x[i];
        y[j] = (T)acc;
    }
}

}  // namespace

fsi_status launch_block_invert(const DevCSR &A, const LevelDev &lev, int storage, int *flags,
                               cudaStream_t s, int num_sms) {
    (void)num_sms;
    if (lev.n_blocks == 0) return FSI_OK;
    const int n = (int)lev.max_block;
    const size_t budget = 200 * 1024;
    int C = 1;
    auto smem_for = [&](int c) {
        const int R = (n + c - 1) / c;
        return ((size_t)R * n + 3 * (size_t)n + R) * sizeof(double);
    };
    while (C < 8 && smem_for(C) > budget) C *= 2;
    if (smem_for(C) > budget) {
        set_error("Schwarz block too large for an 8-CTA cluster (" + std::to_string(n) + " dofs)");
        return FSI_ERR_ARG;
    }
    GJParams P;
    P.blk_ptr = lev.blk_ptr.as<int32_t>();
    P.blk_idx = lev.blk_idx.as<int32_t>();
    P.blk_off = lev.blk_off.as<int64_t>();
    P.row_ptr = A.ptr.as<int32_t>();
    P.col = A.col.as<int32_t>();
    P.val = A.val64.as<double>();
    P.inv = lev.inv.p;
    P.scale = lev.inv_scale.as<float>();
    P.storage = storage;
    P.rows_per_cta = (n + C - 1) / C;
    P.flags = flags;
    const size_t smem = smem_for(C);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(lev.n_blocks * C));
    cfg.blockDim = dim3(GJ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (C) {
        case 1:
            FSI_CUDA(cudaFuncSetAttribute(block_gj_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            FSI_CUDA(cudaLaunchKernelEx(&cfg, block_gj_kernel<1>, P));
            count_launch();
            break;
        case 2:
            FSI_CUDA(cudaFuncSetAttribute(block_gj_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            FSI_CUDA(cudaLaunchKernelEx(&cfg, block_gj_kernel<2>, P));
            count_launch();
            break;
        case 4:
            FSI_CUDA(cudaFuncSetAttribute(block_gj_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            FSI_CUDA(cudaLaunchKernelEx(&cfg, block_gj_kernel<4>, P));
            count_launch();
            break;
        default:
            FSI_CUDA(cudaFuncSetAttribute(block_gj_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            FSI_CUDA(cudaLaunchKernelEx(&cfg, block_gj_kernel<8>, P));
            count_launch();
            break;
    }
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

template <class T>
fsi_status launch_block_apply(const LevelDev &lev, const T *r, T *x, T omega, int transpose, cudaStream_t s,
                              int64_t it0, int64_t it1) {
    // items [it0, it1) (a pass of the multiplicative sweep), or all of them
    const bool ranged = it1 >= 0;
    if (!ranged) { it0 = 0; it1 = lev.n_items; }
    if (it0 < 0 || it1 > lev.n_items || it0 > it1) { set_error("work-item range out of bounds"); return FSI_ERR_ARG; }
    const int64_t n_it = it1 - it0;
    if (n_it == 0) return FSI_OK;
    const int4 *items = lev.items.as<int4>() + it0;
    if (lev.max_block > MAX_BLOCK) {
        set_error("Schwarz block larger than the apply kernel's staging buffer");
        return FSI_ERR_ARG;
    }
    // overlapping blocks (a whole additive level): per-slot results, then the
    // owner-computes combination; a pass of the multiplicative sweep holds
    // disjoint blocks and adds into x directly
    T *stage = (!ranged && lev.n_own > 0) ? lev.stage.as<T>() : nullptr;
    if (std::is_same<T, float>::value && lev.inv_store == 2) {
        const float *rf = reinterpret_cast<const float *>(r);
        float *xf = reinterpret_cast<float *>(x);
        float *sf = reinterpret_cast<float *>(stage);
        if (transpose && lev.max_block <= 256)
            FSI_CUDA(launch_pdl(block_apply_h_tr_kernel, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
                items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
                lev.blk_w.as<float>(), lev.inv.as<__half>(), lev.inv_scale.as<float>(), lev.jac_idx.as<int32_t>(),
                lev.jac_inv.as<float>(), rf, xf, (float)omega, sf));
        else if (transpose)
            FSI_CUDA(launch_pdl(block_apply_h_t_kernel, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
                items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
                lev.blk_w.as<float>(), lev.inv.as<__half>(), lev.inv_scale.as<float>(), lev.jac_idx.as<int32_t>(),
                lev.jac_inv.as<float>(), rf, xf, (float)omega, sf));
        else if (lev.max_block <= 256)
            FSI_CUDA(launch_pdl(block_apply_h_pipe_kernel, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
                items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
                lev.blk_w.as<float>(), lev.inv.as<__half>(), lev.inv_scale.as<float>(), lev.jac_idx.as<int32_t>(),
                lev.jac_inv.as<float>(), rf, xf, (float)omega, sf));
        else
            FSI_CUDA(launch_pdl(block_apply_h_kernel<4>, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
                items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
                lev.blk_w.as<float>(), lev.inv.as<__half>(), lev.inv_scale.as<float>(), lev.jac_idx.as<int32_t>(),
                lev.jac_inv.as<float>(), rf, xf, (float)omega, sf));
    } else if (transpose) {
        FSI_CUDA(launch_pdl(block_apply_t_kernel<T>, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
            items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
            lev.blk_w.as<T>(), lev.inv.as<T>(), lev.jac_idx.as<int32_t>(), lev.jac_inv.as<T>(), r, x, omega, stage));
    } else {
        FSI_CUDA(launch_pdl(block_apply_kernel<T>, dim3((unsigned)n_it), dim3(APPLY_THREADS), 0, s,
            items, lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), lev.blk_off.as<int64_t>(),
            lev.blk_w.as<T>(), lev.inv.as<T>(), lev.jac_idx.as<int32_t>(), lev.jac_inv.as<T>(), r, x, omega, stage));
    }
    count_launch();
    FSI_CUDA(cudaGetLastError());
    if (stage) {
        const unsigned g = (unsigned)((lev.n_own + 255) / 256);
        FSI_CUDA(launch_pdl(block_gather_kernel<T>, dim3(g), dim3(256), 0, s, lev.own_dof.as<int32_t>(),
                            lev.own_ptr.as<int32_t>(), lev.own_pos.as<int32_t>(), lev.own_w.as<T>(), lev.n_own,
                            (const T *)stage, x, omega, transpose ? 0 : 1));
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    return FSI_OK;
}

template <class T>
fsi_status launch_jacobi_apply(const LevelDev &lev, const T *r, T *x, T omega, cudaStream_t s) {
    if (lev.n_jac == 0) return FSI_OK;
    int64_t g = (lev.n_jac + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    jacobi_kernel<T><<<(unsigned)g, 256, 0, s>>>(lev.jac_idx.as<int32_t>(), lev.jac_inv.as<T>(), lev.n_jac, r, x, omega);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

__global__ void transpose_kernel(const double *__restrict__ m, int64_t n, double *__restrict__ t) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n * n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / n, j = k % n;
        t[j * n + i] = m[k];
    }
}

fsi_status launch_transpose(const double *m, int64_t n, double *t, cudaStream_t s) {
    if (n == 0) return FSI_OK;
    transpose_kernel<<<256, 256, 0, s>>>(m, n, t);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status coarse_invert(const DevCSR &A0, int64_t n0, double *inv, int *flags, cudaStream_t s, double *work) {
    // [A | I] -> [I | A^{-1}] in n0 x 2 n0 working storage: the caller's
    // (no allocation, no synchronisation) or a temporary
    DevBuf Mb;
    if (!work) {
        FSI_TRY(Mb.alloc((size_t)n0 * 2 * n0 * 8));
        work = Mb.as<double>();
    }
    double *M = work;
    coarse_init_kernel<<<256, 256, 0, s>>>(nullptr, nullptr, nullptr, n0, M);
    count_launch();
    coarse_fill_kernel<<<64, 256, 0, s>>>(A0.ptr.as<int32_t>(), A0.col.as<int32_t>(), A0.val64.as<double>(), n0,
                                          M);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    for (int64_t k = 0; k < n0; ++k) {
        coarse_pivot_kernel<<<1, 1024, 0, s>>>(M, n0, k, flags);
        count_launch();
        coarse_elim_kernel<<<(unsigned)n0, 256, 0, s>>>(M, n0, k);
        count_launch();
    }
    FSI_CUDA(cudaGetLastError());
    coarse_extract_kernel<<<256, 256, 0, s>>>(M, n0, inv);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    if (Mb.p) FSI_CUDA(cudaStreamSynchronize(s));     // the temporary goes out of scope
    return FSI_OK;
}

template <class T>
fsi_status launch_dense_gemv(const double *M, int64_t n, const T *x, T *y, int transpose, cudaStream_t s) {
    if (transpose) {
        FSI_CUDA(launch_pdl(dense_gemv_t_kernel<T>, dim3((unsigned)((n + 127) / 128)), dim3(128), 0, s, M, n, x, y));
        count_launch();
    } else {
        int64_t blocks = (n * 32 + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        FSI_CUDA(launch_pdl(dense_gemv_kernel<T>, dim3((unsigned)blocks), dim3(256), 0, s, M, n, x, y));
        count_launch();
    }
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

template fsi_status launch_block_apply<float>(const LevelDev &, const float *, float *, float, int, cudaStream_t,
                                             int64_t, int64_t);
template fsi_status launch_block_apply<double>(const LevelDev &, const double *, double *, double, int, cudaStream_t,
                                             int64_t, int64_t);
template fsi_status launch_jacobi_apply<float>(const LevelDev &, const float *, float *, float, cudaStream_t);
template fsi_status launch_jacobi_apply<double>(const LevelDev &, const double *, double *, double, cudaStream_t);
template fsi_status launch_dense_gemv<float>(const double *, int64_t, const float *, float *, int, cudaStream_t);
template fsi_status launch_dense_gemv<double>(const double *, int64_t, const double *, double *, int, cudaStream_t);

}  // namespace fsi
