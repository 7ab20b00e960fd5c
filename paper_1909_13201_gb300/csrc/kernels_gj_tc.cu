// Batched block inversion for the mixed-precision smoothers (Sec. 3.2, "each
// block solved by LU"): blocked Gauss-Jordan in float32 whose rank-32
// trailing updates run on the 5th-generation tensor cores (tcgen05.mma,
// kind::tf32, accumulator in tensor memory).
//
// The block's rows live in shared memory (float32, row-major), split over a
// thread-block cluster of C CTAs when they do not fit one CTA.  Columns are
// eliminated in panels of 32:
//   1. the CTA owning the panel's 32 rows forms Rp = D^{-1} M[K, :] (D =
//      M[K, K]) with the panel columns replaced by D^{-1}: unblocked Gauss-
//      Jordan restricted to the 32 panel rows, the rows held in registers by
//      all eight warps (4 rows x NCH 32-column chunks per thread), one pivot
//      row and one multiplier column published through shared memory per
//      step;
//   2. Rp is written, transposed and rounded to TF32, into the owner's
//      operand buffer; after a cluster barrier the other CTAs copy it over
//      distributed shared memory and arrive on the owner's copy barrier (an
//      mbarrier the owner waits on before it writes its next operand);
//   3. every CTA builds F = -M[rows, K] (zero on the panel rows), zeroes
//      M[rows, K], and one thread issues D_tmem = F x Rp (M = 128 rows per
//      MMA, N <= 256 columns, K = 8 per instruction, 4 instructions);
//   4. the accumulator is read back with tcgen05.ld and added to M.
// After the last panel M holds A^{-1} (unpivoted, as the float64 kernel:
// the J2 order inside a block puts the positive-definite momentum/ALE
// unknowns before the pressures).  The same kernel with TC = false does the
// rank-32 update with float32 FMAs on the CUDA cores (reference variant).
//
// Operand layout (no swizzle): 8-row x 16-byte core matrices; element (r, k)
// of a 32-wide K panel sits at (r/8)*1024 + (k/4)*128 + (r%8)*16 + (k%4)*4
// bytes, so the leading (K) byte offset is 128 and the stride (M/N) byte
// offset 1024; K step s starts 256 s bytes in.  Every wait is bounded.
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include <cublas_v2.h>

#include "context.h"

namespace cg = cooperative_groups;

namespace fsi {

namespace {

constexpr int TC_THREADS = 256;
constexpr int PANEL = 32;
constexpr int CM_SBO = 1024, CM_LBO = 128;
constexpr int NCH_MAX = 16;       // 32-column chunks of a panel row held in registers (n <= 512)
// mbarriers, TMEM slot, flags; the published pivot rows [2][NCH_MAX * 32] and
// multiplier columns [2][PANEL] of the panel step
constexpr size_t MISC_BYTES = 64 + 2 * NCH_MAX * 32 * 4 + 2 * PANEL * 4 + 64;
constexpr int HT = 1024;          // slots of the gather's dof -> position table (> 2 x the largest block)

struct GJTCParams {
    const int32_t *blk_ptr, *blk_idx;
    const int64_t *blk_off;
    const int32_t *row_ptr, *col;
    const double *val;
    void *inv;                 // float or __half
    float *scale;              // float16 storage: per block row
    int storage;               // 1 float32, 2 float16 + row scale
    int n_max;                 // largest block
    int rows_per_cta;          // R (multiple of 32)
    int ldm;                   // row stride of M in shared memory (floats)
    int npad;                  // columns rounded up to 16
    int tiles;                 // 128-row MMA tiles per CTA
    int tmem_cols;             // allocated tensor-memory columns
    size_t off_f, off_b, off_misc;   // shared-memory offsets (bytes)
    int *flags;                // [0] zero pivot, [2] |= 4: MMA wait timed out
    const float *dense;        // dense mode: block b is dense[b n n ..], row-major n x n (every block n = n_max)
};

__host__ __device__ inline int cm_off(int r, int k) {
    return (r >> 3) * CM_SBO + (k >> 2) * CM_LBO + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((CM_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((CM_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                        // descriptor version of this architecture family
    return d;                                      // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// column of chunk c, lane l in the panel step of panel columns [k0, k0 + 32):
// chunk 0 holds the panel columns, chunks 1.. the others in increasing order
__device__ __forceinline__ int panel_col(int c, int l, int k0) {
    if (c == 0) return k0 + l;
    const int jo = 32 * (c - 1) + l;
    return jo < k0 ? jo : jo + PANEL;
}

template <int C, bool TC, int NCH>
__global__ void __launch_bounds__(TC_THREADS, 2) block_gj_tc_kernel(GJTCParams P) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (C > 1) ? (int)cluster.block_rank() : 0;
    const int blk = blockIdx.x / C;
    const int s0 = P.blk_ptr[blk];
    const int n = P.blk_ptr[blk + 1] - s0;
    const int R = P.rows_per_cta, ldm = P.ldm;
    const int r0 = rank * R;
    const int nr = max(0, min(R, n - r0));             // rows held by this CTA
    const int npad = (n + 15) & ~15;
    float *Ms = reinterpret_cast<float *>(smraw);       // [R][ldm]
    unsigned char *Fs = smraw + P.off_f;                // tiles x 16 KB (A operand)
    unsigned char *Bs = smraw + P.off_b;                // npad x 128 B (B operand, Rp^T)
    unsigned char *misc = smraw + P.off_misc;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(misc);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(misc + 8);
    int *sflag = reinterpret_cast<int *>(misc + 12);    // [0] bad pivot, [1] wait timeout
    uint64_t *cbar = reinterpret_cast<uint64_t *>(misc + 24);   // peers' copies of this CTA's operand done
    float *prow = reinterpret_cast<float *>(misc + 64);            // [2][NCH_MAX * 32] pivot rows
    float *pmul = prow + 2 * NCH_MAX * 32;                         // [2][PANEL] multiplier columns
    int32_t *sidx = reinterpret_cast<int32_t *>(misc + MISC_BYTES);   // [n] block indices (sorted)
    int32_t *rb = sidx + ((n + 3) & ~3);                           // [2 R] CSR bounds of the local rows
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    if (TC && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        sflag[0] = 0;
        sflag[1] = 0;
        if (TC) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        if (C > 1) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(cbar)), "r"(C - 1));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    // gather the local rows (float64 CSR -> float32): a warp per row, lanes
    // over its entries (independent global loads), each column's position in
    // the block from an open-addressing table global dof -> local position
    // built in the (not yet used) F buffer
    if (P.dense) {
        // dense mode: the block's rows from a row-major n x n array
        const float *src = P.dense + (size_t)blk * n * n;
        for (int t = tid; t < nr * n; t += blockDim.x) {
            const int li = t / n, c = t - li * n;
            Ms[(size_t)li * ldm + c] = src[(size_t)(r0 + li) * n + c];
        }
        for (int t = tid; t < nr; t += blockDim.x)
            for (int c = n; c < ldm; ++c) Ms[(size_t)t * ldm + c] = 0.f;
    } else {
        int *hkey = reinterpret_cast<int *>(Fs);
        int *hval = hkey + HT;
        for (int t = tid; t < nr * ldm; t += blockDim.x) Ms[t] = 0.f;
        for (int t = tid; t < HT; t += blockDim.x) hkey[t] = -1;
        for (int t = tid; t < n; t += blockDim.x) sidx[t] = P.blk_idx[s0 + t];
        // the CSR bounds of every local row at once (one round trip)
        for (int t = tid; t < nr; t += blockDim.x) {
            const int g = P.blk_idx[s0 + r0 + t];
            rb[2 * t] = P.row_ptr[g];
            rb[2 * t + 1] = P.row_ptr[g + 1];
        }
        __syncthreads();
        for (int t = tid; t < n; t += blockDim.x) {
            const int key = sidx[t];
            uint32_t h = ((uint32_t)key * 0x9E3779B1u) >> 22;            // 10 bits: HT = 1024
            while (true) {                                               // n < HT: an empty slot exists
                const int prev = atomicCAS(&hkey[h], -1, key);
                if (prev == -1) { hval[h] = t; break; }
                h = (h + 1) & (HT - 1);
            }
        }
        __syncthreads();
        // four rows per warp at a time (rows li0 + 8 r), up to 128 entries of
        // each: 16 column indices and 16 values per lane loaded before any is
        // used
        constexpr int NW = TC_THREADS / 32, RG = 4, SUBC = 4;
        for (int li0 = warp; li0 < nr; li0 += RG * NW) {
            int a[RG], b[RG];
            int len = 0;
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const int li = li0 + r * NW;
                a[r] = b[r] = 0;
                if (li < nr) {
                    a[r] = rb[2 * li];
                    b[r] = rb[2 * li + 1];
                }
                len = max(len, b[r] - a[r]);
            }
            for (int off = lane; off < len; off += 32 * SUBC) {
                int cc[SUBC * RG];
                float vv[SUBC * RG];
#pragma unroll
                for (int u = 0; u < SUBC * RG; ++u) {
                    const int r = u / SUBC, k = a[r] + off + 32 * (u % SUBC);
                    const bool in = k < b[r];
                    cc[u] = in ? P.col[k] : -1;
                    vv[u] = in ? (float)P.val[k] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < SUBC * RG; ++u) {
                    const int c = cc[u];
                    if (c < 0) continue;
                    uint32_t h = ((uint32_t)c * 0x9E3779B1u) >> 22;
                    int pos = -1;
                    while (true) {
                        const int kk = hkey[h];
                        if (kk == c) { pos = hval[h]; break; }
                        if (kk == -1) break;
                        h = (h + 1) & (HT - 1);
                    }
                    if (pos >= 0) Ms[(size_t)(li0 + (u / SUBC) * NW) * ldm + pos] = vv[u];
                }
            }
        }
    }
    if (TC) asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (TC) asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = TC ? *tslot : 0u;
    if (C > 1) cluster.sync();

    const int npanels = (n + PANEL - 1) / PANEL;
    constexpr int QN = PANEL / (TC_THREADS / 32);       // consecutive panel rows per thread in the panel step
    static_assert(QN == 4, "the panel step moves 4 rows per thread as float4");
    int owned = 0;                                      // panels this CTA has owned so far
    for (int p = 0; p < npanels; ++p) {
        const int k0 = p * PANEL, kw = min(PANEL, n - k0);
        const int owner = k0 / R;
        const bool own = rank == owner;
        const int lb = k0 - r0;                         // first panel row (local, owner)
        // ---- F = -M[rows, K] (0 on the owner's panel rows) into the A operand,
        //      then M[rows, K] = 0.  Neither touches the panel rows: the other
        //      CTAs do both while they wait for the owner's operand, the owner
        //      after the cluster barrier that releases them.  Thread order of F walks each 8 x 16-byte core matrix
        //      contiguously.
        auto build_f = [&]() {
            constexpr int NE = 128 * PANEL / TC_THREADS;
            for (int tile = 0; tile < P.tiles; ++tile) {
#pragma unroll 4
                for (int i = 0; i < NE; ++i) {
                    const int e = tid + i * TC_THREADS;
                    const int t = (e & 3) | (((e >> 5) & 7) << 2);
                    const int lr = ((e >> 2) & 7) | ((e >> 8) << 3), li = tile * 128 + lr;
                    float v = 0.f;
                    if (li < nr && t < kw && !(own && li >= lb && li < lb + kw)) v = -Ms[(size_t)li * ldm + k0 + t];
                    *reinterpret_cast<float *>(Fs + (size_t)tile * 16384 + cm_off(lr, t)) = TC ? to_tf32(v) : v;
                }
            }
        };
        auto zero_k = [&]() {
            if (lane < kw)
                for (int li = warp; li < nr; li += TC_THREADS / 32)
                    if (!(own && li >= lb && li < lb + kw)) Ms[(size_t)li * ldm + k0 + lane] = 0.f;
        };
        // ---- 1. owner: Gauss-Jordan on the panel rows M[K, :] (steps t < kw,
        //         pivot M[k0 + t, k0 + t]); column k0 + t takes the identity
        //         column before its step, so the panel columns end as D^{-1}.
        //         Thread: rows u = 4 warp + q (q < 4), chunks c < NCH at columns
        //         panel_col(c, lane).  Before step t the warp holding row t
        //         publishes it scaled by 1 / pivot (the pivot's entry replaced by
        //         1 / pivot) and lane t of every warp its multipliers M[u, k0 + t]
        //         (double-buffered: one barrier per step); step t is then one
        //         FMA per held entry.
        if (own) {
            float acc[QN][NCH];
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int u = QN * warp + q;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int j = panel_col(c, lane, k0);
                    acc[q][c] = (u < kw && j < n) ? Ms[(size_t)(lb + u) * ldm + j] : 0.f;
                }
            }
            bool bad = false;
            if (warp == 0) {
                float piv = __shfl_sync(0xffffffffu, acc[0][0], 0);
                if (!(fabsf(piv) > 1e-30f) || !isfinite(piv)) {
                    bad = true;
                    piv = 1.f;
                }
                const float ip = 1.f / piv;
#pragma unroll
                for (int c = 0; c < NCH; ++c) prow[c * 32 + lane] = (c == 0 && lane == 0) ? ip : acc[0][c] * ip;
            }
            if (lane == 0)
                *reinterpret_cast<float4 *>(pmul + QN * warp) = make_float4(acc[0][0], acc[1][0], acc[2][0], acc[3][0]);
            __syncthreads();
#pragma unroll
            for (int t = 0; t < PANEL; ++t) {
                if (t < kw) {
                    const float *pr = prow + (t & 1) * NCH_MAX * 32;
                    const float4 f4 = *reinterpret_cast<const float4 *>(pmul + (t & 1) * PANEL + QN * warp);
                    const float f[QN] = {f4.x, f4.y, f4.z, f4.w};
                    float sv[NCH];
#pragma unroll
                    for (int c = 0; c < NCH; ++c) sv[c] = pr[c * 32 + lane];
#pragma unroll
                    for (int q = 0; q < QN; ++q) {
                        acc[q][0] = fmaf(-f[q], sv[0], lane == t ? 0.f : acc[q][0]);
#pragma unroll
                        for (int c = 1; c < NCH; ++c) acc[q][c] = fmaf(-f[q], sv[c], acc[q][c]);
                    }
                    if (warp == t / QN)
#pragma unroll
                        for (int c = 0; c < NCH; ++c) acc[t % QN][c] = sv[c];
                    const int t1 = t + 1;
                    if (t1 < kw) {
                        float *nrow = prow + (t1 & 1) * NCH_MAX * 32;
                        if (warp == t1 / QN) {
                            float piv = __shfl_sync(0xffffffffu, acc[t1 % QN][0], t1 % 32);
                            if (!(fabsf(piv) > 1e-30f) || !isfinite(piv)) {
                                bad = true;
                                piv = 1.f;
                            }
                            const float ip = 1.f / piv;
#pragma unroll
                            for (int c = 0; c < NCH; ++c)
                                nrow[c * 32 + lane] = (c == 0 && lane == t1) ? ip : acc[t1 % QN][c] * ip;
                        }
                        if (lane == t1)
                            *reinterpret_cast<float4 *>(pmul + (t1 & 1) * PANEL + QN * warp) =
                                make_float4(acc[0][0], acc[1][0], acc[2][0], acc[3][0]);
                        __syncthreads();
                    }
                }
            }
            if (bad) sflag[0] = 1;
            // ---- 2. the other CTAs finished copying this CTA's previous
            //         operand (bounded wait on the copy barrier's phase), then
            //         Rp back into the panel rows and Rp^T (TF32, zero-padded to
            //         32 x npad) into the B buffer, 4 rows per 16-byte store
            if (C > 1 && owned > 0 && !sflag[1]) {     // after a timed-out wait no further waits
                uint32_t done = 0;
                for (int it = 0; it < (1 << 20) && !done; ++it) {
                    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 q, [%1], %2;\n"
                                 "selp.u32 %0, 1, 0, q;\n}"
                                 : "=r"(done)
                                 : "r"(smem_u32(cbar)), "r"((uint32_t)((owned - 1) & 1))
                                 : "memory");
                }
                if (!done) sflag[1] = 1;
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int j = panel_col(c, lane, k0);
                float w[QN];
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    const int u = QN * warp + q;
                    const bool live = u < kw && j < n;
                    if (live) Ms[(size_t)(lb + u) * ldm + j] = acc[q][c];
                    w[q] = live ? (TC ? to_tf32(acc[q][c]) : acc[q][c]) : 0.f;
                }
                if (j < npad) *reinterpret_cast<float4 *>(Bs + cm_off(j, QN * warp)) = make_float4(w[0], w[1], w[2], w[3]);
            }
            ++owned;
        } else {
            build_f();
            __syncthreads();
            zero_k();
        }
        if (C > 1) {
            cluster.sync();
            // the other CTAs copy the owner's operand (16-byte DSMEM reads, in
            // parallel), then one thread each arrives on the owner's copy barrier
            if (rank != owner) {
                const float4 *src = reinterpret_cast<const float4 *>(cluster.map_shared_rank(Bs, owner));
                float4 *dstp = reinterpret_cast<float4 *>(Bs);
                for (int e = tid; e < npad * PANEL / 4; e += blockDim.x) dstp[e] = src[e];
            }
        }
        __syncthreads();
        if (C > 1 && rank != owner && tid == 0) {
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(cbar)), "r"(owner));
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
        }
        // after the last operand copy no CTA touches another's shared memory:
        // arrive on the cluster barrier now, wait for it only before exit
        if (C > 1 && p == npanels - 1) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        // the owner builds its A operand once the other CTAs are released
        if (own) {
            build_f();
            __syncthreads();
            zero_k();
        }
        if (TC) {
            // ---- 4a. tensor cores: D = F x Rp, then M += D
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                const int nchunks = (npad + 255) / 256;
                const int nc = ((npad / nchunks) + 15) & ~15;
                for (int tile = 0; tile < P.tiles; ++tile) {
                    for (int ch = 0; ch < nchunks; ++ch) {
                        const int c0 = ch * nc, cw = min(nc, npad - c0);
                        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(cw >> 3) << 17) |
                                               ((uint32_t)(128 >> 4) << 24);
                        const uint32_t dt = tmem + (uint32_t)(tile * npad + c0);
                        const uint32_t a0 = smem_u32(Fs + (size_t)tile * 16384);
                        const uint32_t b0 = smem_u32(Bs + (size_t)(c0 >> 3) * CM_SBO);
                        for (int s = 0; s < PANEL / 8; ++s) {
                            const uint64_t ad = smem_desc(a0 + s * 2 * CM_LBO);
                            const uint64_t bd = smem_desc(b0 + s * 2 * CM_LBO);
                            const uint32_t acc = s > 0 ? 1u : 0u;
                            asm volatile("{\n.reg .pred q;\nsetp.ne.u32 q, %4, 0;\n"
                                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(dt),
                                         "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(mbar)));
            }
            {
                uint32_t done = 0;
                for (int it = 0; it < (1 << 20) && !done; ++it) {
                    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                                 "selp.u32 %0, 1, 0, q;\n}"
                                 : "=r"(done)
                                 : "r"(smem_u32(mbar)), "r"((uint32_t)(p & 1)));
                }
                if (!done) sflag[1] = 1;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // each warp reads its 32-lane quarter; the two warps of a quarter split the columns
            const int q = warp & 3, half = warp >> 2;
            for (int tile = 0; tile < P.tiles; ++tile) {
                const int li = tile * 128 + q * 32 + lane;
                for (int c0 = half * 16; c0 < npad; c0 += 32) {
                    uint32_t v[16];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tile * npad + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (li < nr) {
                        float *mrow = Ms + (size_t)li * ldm;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < n) mrow[c0 + j] += __uint_as_float(v[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        } else {
            // ---- 4b. CUDA cores: M[i, :] += F[i, :] x Rp (float32 FMAs)
            __syncthreads();
            for (int e = tid; e < nr * n; e += blockDim.x) {
                const int li = e / n, j = e - li * n;
                const unsigned char *frow = Fs + (size_t)(li >> 7) * 16384;
                float acc = 0.f;
#pragma unroll 8
                for (int t = 0; t < PANEL; ++t)
                    acc = fmaf(*reinterpret_cast<const float *>(frow + cm_off(li & 127, t)),
                               *reinterpret_cast<const float *>(Bs + cm_off(j, t)), acc);
                Ms[(size_t)li * ldm + j] += acc;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        if (sflag[0]) atomicExch(P.flags, 1);
        if (sflag[1]) atomicOr(P.flags + 2, 4);
    }
    // ---- output
    const int64_t off = P.blk_off[blk];
    if (P.storage == 2) {
        const int ldo = (n + 7) & ~7;
        __half *out = static_cast<__half *>(P.inv) + off;
        for (int li = warp; li < nr; li += TC_THREADS / 32) {
            float m = 0.f;
            for (int j = lane; j < n; j += 32) m = fmaxf(m, fabsf(Ms[(size_t)li * ldm + j]));
            m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));   // m >= 0
            const float sc = m > 0.f ? m : 1.f;
            if (lane == 0) P.scale[s0 + r0 + li] = sc;
            const float isc = 1.f / sc;
            for (int j = lane; j < ldo; j += 32)
                out[(size_t)(r0 + li) * ldo + j] = __float2half_rn(j < n ? Ms[(size_t)li * ldm + j] * isc : 0.f);
        }
    } else {
        const int ldo = (n + 3) & ~3;
        float *out = static_cast<float *>(P.inv) + off;
        for (int t = tid; t < nr * ldo; t += blockDim.x) {
            const int li = t / ldo, j = t - li * ldo;
            out[(size_t)(r0 + li) * ldo + j] = (j < n) ? Ms[(size_t)li * ldm + j] : 0.f;
        }
    }
    if (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols));
    }
    if (C > 1) {
        if (npanels == 0) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

template <int C, bool TC, int NCH>
fsi_status launch_tc(const GJTCParams &P, int64_t n_blocks, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_blocks * C));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FSI_CUDA(cudaFuncSetAttribute(block_gj_tc_kernel<C, TC, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FSI_CUDA(cudaLaunchKernelEx(&cfg, block_gj_tc_kernel<C, TC, NCH>, P));
    count_launch();
    return FSI_OK;
}

// The kernel for blocks of up to n dofs in clusters of C CTAs: a panel row
// of n columns takes NCH = ceil(n / 32) register chunks, rounded up to 6, 12
// or 16.  Instantiated for the (NCH, C) pairs gj_tc_plan yields for n <= 512:
// (6, 1) n <= 128, (6, 2) up to 176, (6, 4) up to 192, (12, 4) up to 384
// except (12, 8) for 240..256, (16, 8) up to 512.
template <bool TC>
fsi_status launch_gj(const GJTCParams &P, int n, int C, int64_t n_blocks, size_t smem, cudaStream_t s) {
    const int nch = n <= 6 * 32 ? 6 : n <= 12 * 32 ? 12 : 16;
    if (nch == 6 && C == 1) return launch_tc<1, TC, 6>(P, n_blocks, smem, s);
    if (nch == 6 && C == 2) return launch_tc<2, TC, 6>(P, n_blocks, smem, s);
    if (nch == 6 && C == 4) return launch_tc<4, TC, 6>(P, n_blocks, smem, s);
    if (nch == 12 && C == 4) return launch_tc<4, TC, 12>(P, n_blocks, smem, s);
    if (nch == 12 && C == 8) return launch_tc<8, TC, 12>(P, n_blocks, smem, s);
    if (nch == 16 && C == 8) return launch_tc<8, TC, 16>(P, n_blocks, smem, s);
    set_error("no block inversion kernel for blocks of " + std::to_string(n) + " dofs in clusters of " +
              std::to_string(C));
    return FSI_ERR_ARG;
}

}  // namespace

// Shared-memory and tensor-memory plan for blocks of up to n dofs.  First
// choice: the smallest cluster whose CTAs fit two to an SM (<= 112 KB of
// shared memory, <= 256 tensor-memory columns each, so two co-resident CTAs
// -- of one cluster or two -- never wait on each other's columns): while one
// CTA is in a serial panel step the other keeps the SM busy.  Otherwise the
// smallest cluster that fits at all, one CTA per SM (a cluster's CTAs then
// never share an SM: a second CTA waiting in tcgen05.alloc behind the
// first's columns would never proceed).  Rows are stored with an odd stride,
// so a warp reading one column of 32 consecutive rows hits 32 banks.
static size_t gj_tc_bytes(int n, int C, int R, int *cols_out) {
    const int npad = (n + 15) & ~15;
    const int tiles = (R + 127) / 128;
    int cols = 32;
    while (cols < tiles * npad) cols *= 2;
    *cols_out = tiles * npad > 512 ? 1 << 30 : cols;
    const int ldm = n | 1;
    const size_t m_bytes = ((size_t)R * ldm * 4 + 1023) & ~(size_t)1023;
    const size_t f_bytes = (size_t)tiles * 16384;
    const size_t b_bytes = ((size_t)npad * 128 + 1023) & ~(size_t)1023;
    // misc: barrier, flags, Dm; then the block's indices and the row offsets
    return m_bytes + f_bytes + b_bytes + MISC_BYTES + (size_t)(((n + 3) & ~3) + 2 * R + 4) * 4;
}

bool gj_tc_plan(int n, int *C_out, int *R_out, size_t *smem_out) {
    for (int pass = 0; pass < 2; ++pass) {
        const size_t budget = pass == 0 ? 112 * 1024 : 225 * 1024;
        for (int C = 1; C <= 8; C *= 2) {
            int R = (n + C - 1) / C;
            if (C > 1) R = (R + PANEL - 1) / PANEL * PANEL;
            int cols = 0;
            size_t total = gj_tc_bytes(n, C, R, &cols);
            if (cols > 512) continue;
            if (pass == 0 && cols > 256) continue;
            if (pass == 1 && C > 1) total = std::max(total, (size_t)120 * 1024);
            if (total <= budget) {
                *C_out = C;
                *R_out = R;
                *smem_out = total;
                return true;
            }
        }
    }
    return false;
}

fsi_status launch_block_invert_tc(const DevCSR &A, const LevelDev &lev, int storage, bool tensor, int *flags,
                                  cudaStream_t s) {
    if (lev.n_blocks == 0) return FSI_OK;
    if (storage != 1 && storage != 2) { set_error("float32 block inversion stores float32 or float16"); return FSI_ERR_ARG; }
    const int n = (int)lev.max_block;
    int C = 1, R = 0;
    size_t smem = 0;
    if (!gj_tc_plan(n, &C, &R, &smem)) {
        set_error("Schwarz block too large for the float32 cluster inversion (" + std::to_string(n) + " dofs)");
        return FSI_ERR_ARG;
    }
    GJTCParams P;
    P.blk_ptr = lev.blk_ptr.as<int32_t>();
    P.blk_idx = lev.blk_idx.as<int32_t>();
    P.blk_off = lev.blk_off.as<int64_t>();
    P.row_ptr = A.ptr.as<int32_t>();
    P.col = A.col.as<int32_t>();
    P.val = A.val64.as<double>();
    P.inv = lev.inv.p;
    P.scale = lev.inv_scale.as<float>();
    P.storage = storage;
    P.n_max = n;
    P.rows_per_cta = R;
    const int ldm = n | 1;
    P.ldm = ldm;
    P.npad = (n + 15) & ~15;
    P.tiles = (R + 127) / 128;
    int cols = 32;
    while (cols < P.tiles * P.npad) cols *= 2;
    P.tmem_cols = cols;
    P.off_f = ((size_t)R * ldm * 4 + 1023) & ~(size_t)1023;
    P.off_b = P.off_f + (size_t)P.tiles * 16384;
    P.off_misc = P.off_b + (((size_t)P.npad * 128 + 1023) & ~(size_t)1023);
    P.flags = flags;
    P.dense = nullptr;
    return tensor ? launch_gj<true>(P, n, C, lev.n_blocks, smem, s) : launch_gj<false>(P, n, C, lev.n_blocks, smem, s);
}

// ---------------------------------------------------------------------------
// Monolithic Schwarz blocks larger than one cluster holds (the AS comparison
// preconditioner in 3D: all fields of the closure of 8 hexahedra, ~750
// dofs).  The block's unknowns split, in their J2 order, into the
// displacement system (d^s, d^f, p^s: a prefix of the sorted index list) and
// the velocity system (u^s, u^f, p^f); with M = [A B; C D] on that split,
//   X = A^{-1},  S = D - C X B,  Y = S^{-1},
//   M^{-1} = [X + X B Y C X, -X B Y; -Y C X, Y],
// evaluated as U = C X, T = X B, S = D - U B, Y = S^{-1}, TR = -T Y,
// BL = -Y U, TL = X - T BL.  A and S (each about half the block) are
// inverted by the cluster Gauss-Jordan kernel in dense mode, the products
// are float32 batched GEMMs (cuBLAS).  Every block is padded to the
// largest split sizes N1, N2 with identity rows and columns (the padded M is
// blockdiag(M, I), whose inverse is blockdiag(M^{-1}, I)), so a chunk of
// blocks is one strided batch.

// A, B, C, D of blocks [j0, j0 + gridDim.x) from the CSR, padded; zeroed first
__global__ void __launch_bounds__(256) schur_gather_kernel(const int32_t *__restrict__ row_ptr,
                                                            const int32_t *__restrict__ col,
                                                            const double *__restrict__ val,
                                                            const int32_t *__restrict__ blk_ptr,
                                                            const int32_t *__restrict__ blk_idx, int64_t j0,
                                                            int off3, int N1, int N2, float *__restrict__ Ad,
                                                            float *__restrict__ Bd, float *__restrict__ Cd,
                                                            float *__restrict__ Dd) {
    constexpr int HT2 = 2048;
    __shared__ int hkey[HT2], hval[HT2];
    const int64_t j = j0 + blockIdx.x;
    const int s0 = blk_ptr[j], n = blk_ptr[j + 1] - s0;
    float *A = Ad + (size_t)blockIdx.x * N1 * N1, *B = Bd + (size_t)blockIdx.x * N1 * N2;
    float *C = Cd + (size_t)blockIdx.x * N2 * N1, *D = Dd + (size_t)blockIdx.x * N2 * N2;
    for (int t = threadIdx.x; t < HT2; t += blockDim.x) hkey[t] = -1;
    __shared__ int n1s;
    if (threadIdx.x == 0) n1s = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int key = blk_idx[s0 + t];
        if (key < off3) atomicAdd(&n1s, 1);
        uint32_t h = ((uint32_t)key * 0x9E3779B1u) >> 21;            // 11 bits
        while (true) {
            const int prev = atomicCAS(&hkey[h], -1, key);
            if (prev == -1) { hval[h] = t; break; }
            h = (h + 1) & (HT2 - 1);
        }
    }
    __syncthreads();
    const int n1 = n1s, n2 = n - n1;
    // zero, then the padding diagonals
    for (int t = threadIdx.x; t < N1 * N1; t += blockDim.x) A[t] = 0.f;
    for (int t = threadIdx.x; t < N1 * N2; t += blockDim.x) B[t] = 0.f;
    for (int t = threadIdx.x; t < N2 * N1; t += blockDim.x) C[t] = 0.f;
    for (int t = threadIdx.x; t < N2 * N2; t += blockDim.x) D[t] = 0.f;
    __syncthreads();
    for (int t = n1 + threadIdx.x; t < N1; t += blockDim.x) A[(size_t)t * N1 + t] = 1.f;
    for (int t = n2 + threadIdx.x; t < N2; t += blockDim.x) D[(size_t)t * N2 + t] = 1.f;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int li = warp; li < n; li += blockDim.x / 32) {
        const int g = blk_idx[s0 + li];
        for (int k = row_ptr[g] + lane; k < row_ptr[g + 1]; k += 32) {
            const int c = col[k];
            uint32_t h = ((uint32_t)c * 0x9E3779B1u) >> 21;
            int pos = -1;
            while (true) {
                const int kk = hkey[h];
                if (kk == c) { pos = hval[h]; break; }
                if (kk == -1) break;
                h = (h + 1) & (HT2 - 1);
            }
            if (pos < 0) continue;
            const float v = (float)val[k];
            if (li < n1) {
                if (pos < n1) A[(size_t)li * N1 + pos] = v;
                else B[(size_t)li * N2 + (pos - n1)] = v;
            } else {
                if (pos < n1) C[(size_t)(li - n1) * N1 + pos] = v;
                else D[(size_t)(li - n1) * N2 + (pos - n1)] = v;
            }
        }
    }
}

// the block's inverse from its four padded parts into the level's storage
// (row-major, rows padded to 4 floats, at blk_off[j])
__global__ void __launch_bounds__(256) schur_scatter_kernel(const int32_t *__restrict__ blk_ptr,
                                                             const int32_t *__restrict__ blk_idx,
                                                             const int64_t *__restrict__ blk_off, int64_t j0,
                                                             int off3, int N1, int N2, const float *__restrict__ TL,
                                                             const float *__restrict__ TR, const float *__restrict__ BL,
                                                             const float *__restrict__ Y, float *__restrict__ inv) {
    const int64_t j = j0 + blockIdx.x;
    const int s0 = blk_ptr[j], n = blk_ptr[j + 1] - s0;
    __shared__ int n1s;
    if (threadIdx.x == 0) n1s = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        if (blk_idx[s0 + t] < off3) atomicAdd(&n1s, 1);
    __syncthreads();
    const int n1 = n1s;
    const int ldo = (n + 3) & ~3;
    float *out = inv + blk_off[j];
    const size_t b = blockIdx.x;
    for (int t = threadIdx.x; t < n * ldo; t += blockDim.x) {
        const int r = t / ldo, c = t - r * ldo;
        float v = 0.f;
        if (c < n) {
            if (r < n1) v = c < n1 ? TL[b * N1 * N1 + (size_t)r * N1 + c] : TR[b * N1 * N2 + (size_t)r * N2 + (c - n1)];
            else v = c < n1 ? BL[b * N2 * N1 + (size_t)(r - n1) * N1 + c]
                            : Y[b * N2 * N2 + (size_t)(r - n1) * N2 + (c - n1)];
        }
        out[(size_t)r * ldo + c] = v;
    }
}

namespace {
// row-major C (m x n) = alpha A (m x k) B (k x n) + beta C, strided batch
// (cuBLAS is column-major: C^T = B^T A^T)
cublasStatus_t sgemm_rm(cublasHandle_t h, int m, int n, int k, float alpha, const float *A, long long sA,
                        const float *B, long long sB, float beta, float *C, long long sC, int batch) {
    return cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, k, &alpha, B, n, sB, A, k, sA, &beta, C, n,
                                     sC, batch);
}

// nb dense row-major N x N matrices at `in` inverted into `out` (float32)
fsi_status invert_dense(const float *in, float *out, int64_t nb, int N, bool tensor, int *flags,
                        const int32_t *dptr, const int64_t *doff, cudaStream_t s) {
    int C = 1, R = 0;
    size_t smem = 0;
    if (!gj_tc_plan(N, &C, &R, &smem)) {
        set_error("Schur part too large for the cluster inversion (" + std::to_string(N) + ")");
        return FSI_ERR_ARG;
    }
    GJTCParams P;
    P.blk_ptr = dptr;
    P.blk_idx = nullptr;
    P.blk_off = doff;
    P.row_ptr = nullptr;
    P.col = nullptr;
    P.val = nullptr;
    P.inv = out;
    P.scale = nullptr;
    P.storage = 1;
    P.n_max = N;
    P.rows_per_cta = R;
    const int ldm = N | 1;
    P.ldm = ldm;
    P.npad = (N + 15) & ~15;
    P.tiles = (R + 127) / 128;
    int cols = 32;
    while (cols < P.tiles * P.npad) cols *= 2;
    P.tmem_cols = cols;
    P.off_f = ((size_t)R * ldm * 4 + 1023) & ~(size_t)1023;
    P.off_b = P.off_f + (size_t)P.tiles * 16384;
    P.off_misc = P.off_b + (((size_t)P.npad * 128 + 1023) & ~(size_t)1023);
    P.flags = flags;
    P.dense = in;
    return tensor ? launch_gj<true>(P, N, C, nb, smem, s) : launch_gj<false>(P, N, C, nb, smem, s);
}
}  // namespace

#define FSI_CUBLAS(call)                                                                      \
    do {                                                                                      \
        cublasStatus_t e_ = (call);                                                           \
        if (e_ != CUBLAS_STATUS_SUCCESS) {                                                    \
            set_error(std::string(#call) + " failed (cuBLAS status " + std::to_string((int)e_) + ")"); \
            return FSI_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

fsi_status launch_block_invert_schur(Context &cx, const DevCSR &A, const LevelDev &lev, int64_t off3, bool tensor,
                                     int *flags, cudaStream_t s) {
    if (lev.n_blocks == 0) return FSI_OK;
    if (lev.inv_store != 1) { set_error("the split block inversion stores float32 inverses"); return FSI_ERR_ARG; }
    int n1max = 1, n2max = 1;
    for (int64_t j = 0; j < lev.n_blocks; ++j) {
        int n1 = 0;
        for (int64_t k = lev.h_blk_ptr[j]; k < lev.h_blk_ptr[j + 1]; ++k) n1 += lev.h_blk_idx[k] < off3 ? 1 : 0;
        n1max = std::max(n1max, n1);
        n2max = std::max(n2max, (int)(lev.h_blk_ptr[j + 1] - lev.h_blk_ptr[j]) - n1);
    }
    const int N1 = (n1max + 3) & ~3, N2 = (n2max + 3) & ~3;
    int Ct, Rt;
    size_t sm;
    if (!gj_tc_plan(N1, &Ct, &Rt, &sm) || !gj_tc_plan(N2, &Ct, &Rt, &sm)) {
        set_error("Schwarz block halves too large for the cluster inversion (" + std::to_string(n1max) + ", " +
                  std::to_string(n2max) + " dofs)");
        return FSI_ERR_ARG;
    }
    if (!cx.cublas) {
        cublasHandle_t h = nullptr;
        FSI_CUBLAS(cublasCreate(&h));
        cx.cublas = h;
    }
    cublasHandle_t h = static_cast<cublasHandle_t>(cx.cublas);
    FSI_CUBLAS(cublasSetStream(h, s));
    FSI_CUBLAS(cublasSetMathMode(h, tensor ? CUBLAS_TF32_TENSOR_OP_MATH : CUBLAS_DEFAULT_MATH));
    const size_t q11 = (size_t)N1 * N1, q12 = (size_t)N1 * N2, q22 = (size_t)N2 * N2;
    const size_t per_block = (3 * q11 + 6 * q12 + 2 * q22) * 4;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(lev.n_blocks, ((int64_t)4 << 30) / (int64_t)per_block));
    DevBuf Ad, Bd, Cd, Dd, X, T, U, Y, TR, BL, TL, p1, o1, p2, o2;
    FSI_TRY(Ad.alloc(chunk * q11 * 4));
    FSI_TRY(X.alloc(chunk * q11 * 4));
    FSI_TRY(TL.alloc(chunk * q11 * 4));
    FSI_TRY(Bd.alloc(chunk * q12 * 4));
    FSI_TRY(T.alloc(chunk * q12 * 4));
    FSI_TRY(TR.alloc(chunk * q12 * 4));
    FSI_TRY(Cd.alloc(chunk * q12 * 4));
    FSI_TRY(U.alloc(chunk * q12 * 4));
    FSI_TRY(BL.alloc(chunk * q12 * 4));
    FSI_TRY(Dd.alloc(chunk * q22 * 4));
    FSI_TRY(Y.alloc(chunk * q22 * 4));
    {
        std::vector<int32_t> a(chunk + 1), c(chunk + 1);
        std::vector<int64_t> b(chunk), d(chunk);
        for (int64_t i = 0; i <= chunk; ++i) {
            a[i] = (int32_t)(i * N1);
            c[i] = (int32_t)(i * N2);
        }
        for (int64_t i = 0; i < chunk; ++i) {
            b[i] = i * (int64_t)q11;
            d[i] = i * (int64_t)q22;
        }
        FSI_TRY(p1.alloc(a.size() * 4));
        FSI_TRY(p2.alloc(c.size() * 4));
        FSI_TRY(o1.alloc(b.size() * 8));
        FSI_TRY(o2.alloc(d.size() * 8));
        FSI_CUDA(cudaMemcpyAsync(p1.p, a.data(), a.size() * 4, cudaMemcpyHostToDevice, s));
        FSI_CUDA(cudaMemcpyAsync(p2.p, c.data(), c.size() * 4, cudaMemcpyHostToDevice, s));
        FSI_CUDA(cudaMemcpyAsync(o1.p, b.data(), b.size() * 8, cudaMemcpyHostToDevice, s));
        FSI_CUDA(cudaMemcpyAsync(o2.p, d.data(), d.size() * 8, cudaMemcpyHostToDevice, s));
        FSI_CUDA(cudaStreamSynchronize(s));
    }
    for (int64_t j0 = 0; j0 < lev.n_blocks; j0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, lev.n_blocks - j0);
        schur_gather_kernel<<<nb, 256, 0, s>>>(A.ptr.as<int32_t>(), A.col.as<int32_t>(), A.val64.as<double>(),
                                               lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(), j0, (int)off3,
                                               N1, N2, Ad.as<float>(), Bd.as<float>(), Cd.as<float>(), Dd.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
        FSI_TRY(invert_dense(Ad.as<float>(), X.as<float>(), nb, N1, tensor, flags, p1.as<int32_t>(), o1.as<int64_t>(), s));
        FSI_CUBLAS(sgemm_rm(h, N2, N1, N1, 1.f, Cd.as<float>(), q12, X.as<float>(), q11, 0.f, U.as<float>(), q12, nb));
        FSI_CUBLAS(sgemm_rm(h, N1, N2, N1, 1.f, X.as<float>(), q11, Bd.as<float>(), q12, 0.f, T.as<float>(), q12, nb));
        FSI_CUBLAS(sgemm_rm(h, N2, N2, N1, -1.f, U.as<float>(), q12, Bd.as<float>(), q12, 1.f, Dd.as<float>(), q22, nb));
        FSI_TRY(invert_dense(Dd.as<float>(), Y.as<float>(), nb, N2, tensor, flags, p2.as<int32_t>(), o2.as<int64_t>(), s));
        FSI_CUBLAS(sgemm_rm(h, N1, N2, N2, -1.f, T.as<float>(), q12, Y.as<float>(), q22, 0.f, TR.as<float>(), q12, nb));
        FSI_CUBLAS(sgemm_rm(h, N2, N1, N2, -1.f, Y.as<float>(), q22, U.as<float>(), q12, 0.f, BL.as<float>(), q12, nb));
        FSI_CUDA(cudaMemcpyAsync(TL.p, X.p, (size_t)nb * q11 * 4, cudaMemcpyDeviceToDevice, s));
        FSI_CUBLAS(sgemm_rm(h, N1, N1, N2, -1.f, T.as<float>(), q12, BL.as<float>(), q12, 1.f, TL.as<float>(), q11, nb));
        schur_scatter_kernel<<<nb, 256, 0, s>>>(lev.blk_ptr.as<int32_t>(), lev.blk_idx.as<int32_t>(),
                                                lev.blk_off.as<int64_t>(), j0, (int)off3, N1, N2, TL.as<float>(),
                                                TR.as<float>(), BL.as<float>(), Y.as<float>(), lev.inv.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

}  // namespace fsi
