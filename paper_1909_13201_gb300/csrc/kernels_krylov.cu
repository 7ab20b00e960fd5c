// Flexible GMRES kernels (outer Krylov solver, Sec. 3.2), all float64.
// They serve both the host-driven loop (column index passed by value) and
// the device-driven loop (column index read from the control block, loop
// conditions set with cudaGraphSetConditional inside the solve graph).
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2) in three fused
// streaming passes over the basis V (column-major, one vector per column):
//   pass 1: partial dots V^T w                       (launch_mdot)
//   pass 2: w -= V h1 and partial dots V^T w         (launch_update_dot)
//   pass 3: w -= V h2 and partial ||w||^2            (launch_update_dot, norm_only)
// Each pass writes one partial sum per CTA and vector; a one-CTA kernel adds
// them in a fixed order (deterministic).  The Givens update of the Hessenberg
// column and the residual estimate run in one thread on the device.
#include <algorithm>

#include "context.h"

namespace fsi {

namespace {

constexpr int KMAX = 65;     // vectors in a pass: restart + 1 <= 65
constexpr int KT = 256;      // threads per CTA

constexpr int KW = KT / 32;  // warps per CTA

// Rows are split into gridDim.x contiguous chunks; a CTA walks its chunk in
// tiles of KT rows.  Dot products against the basis are split by vector, not
// by row: vector i belongs to warp i % KW, whose lanes stride over the tile's
// rows (coalesced column reads), so a thread holds ceil(NV / KW) accumulators
// instead of NV and the kernels keep several CTAs per SM.  Each vector's
// partial sum comes from exactly one warp: a fixed shuffle tree, no atomics.
template <int NV> struct Slots { static constexpr int U = (NV + KW - 1) / KW; };

// acc[u] += sum over the tile rows of V[i, r] * ws[r - t0], i = warp + KW u
template <int NV, class TV, class TA>
__device__ __forceinline__ void tile_dots(const TV *__restrict__ V, int64_t ld, int nv, int64_t t0, int64_t r1,
                                          const TA *ws, TA (&acc)[Slots<NV>::U]) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int u = 0; u < Slots<NV>::U; ++u) {
        const int i = warp + KW * u;
        if (i >= nv) break;
        const TV *col = V + (size_t)i * ld;
        TA a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < KT / 32; k += 2) {
            const int64_t ra = t0 + lane + 32 * k, rb = ra + 32;
            if (ra < r1) a0 += (TA)__ldg(col + ra) * ws[lane + 32 * k];
            if (rb < r1) a1 += (TA)__ldg(col + rb) * ws[lane + 32 * (k + 1)];
        }
        acc[u] += a0 + a1;
    }
}

// partials[i] = warp-sum of acc for the warp's vectors
template <int NV, class TA>
__device__ __forceinline__ void store_slot_partials(TA (&acc)[Slots<NV>::U], int nv, double *out) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int u = 0; u < Slots<NV>::U; ++u) {
        const int i = warp + KW * u;
        if (i >= nv) break;
        double v = (double)acc[u];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) out[i] = v;
    }
}

// out[0] = CTA sum of one value per thread (warp trees, then warps in order)
__device__ __forceinline__ void store_cta_sum(double v, double *out) {
    __shared__ double red[KW];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < KW; ++k) s += red[k];
        out[0] = s;
    }
}

// Few vectors (NV <= 8): every thread keeps all NV sums of its rows (a warp
// per vector would leave most warps idle); out[i] = CTA sum of acc[i],
// warp trees then warps in order.
template <int NV>
__device__ __forceinline__ void store_row_partials(double (&acc)[NV], int nv, double *out) {
    __shared__ double red[KW][NV];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i >= nv) break;
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < KW; ++k) v += red[k][i];
        out[i] = v;
    }
}

// Pass 1: partial dots V^T w, streamed without barriers.  TV is the basis
// type (float64, or the float32 copy in the mixed modes, where w is rounded
// to float32 and products and sums are float32), TA the accumulator.
// NV <= 8: a thread keeps all NV sums of its rows and loads 4 rows per pass;
// otherwise vector i belongs to warp i % KW, whose lanes take the rows of the
// CTA's chunk 8 x 32 (float64 basis: 4 x 32) at a time (w is re-read from L1
// by every warp).  Either way a lane has 4 (NV + 1) or 8 (Slots + 1)
// independent loads in flight:
// each pass of the loop costs one memory latency, so the bytes a pass keeps
// in flight (and the CTAs per SM) set the bandwidth.
template <int NV, class TV, class TA>
__device__ __forceinline__ void stream_dots(const TV *__restrict__ V, int64_t ld, int nv,
                                            const double *__restrict__ w, int64_t r0, int64_t r1,
                                            double *__restrict__ out) {
    if constexpr (NV <= 8) {
        TA acc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += 4 * KT) {
            TA wr[4];
            TV v[4][NV];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t rq = r + (int64_t)q * KT;
                wr[q] = rq < r1 ? (TA)__ldg(w + rq) : TA(0);
#pragma unroll
                for (int i = 0; i < NV; ++i) v[q][i] = (i < nv && rq < r1) ? __ldg(V + (size_t)i * ld + rq) : TV(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] += (TA)v[q][i] * wr[q];
        }
        double accd[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) accd[i] = (double)acc[i];
        store_row_partials<NV>(accd, nv, out);
    } else {
        constexpr int U = Slots<NV>::U;
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
        TA acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = 0;
        constexpr int RB = sizeof(TV) == 4 ? 8 : 4;  // row batches of 32 per pass
        for (int64_t r = r0 + lane; r < r1; r += 32 * RB) {
            TA wr[RB];
            TV v[U][RB];
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                const int64_t rq = r + 32 * q;
                wr[q] = rq < r1 ? (TA)__ldg(w + rq) : TA(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = warp + KW * u;
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int64_t rq = r + 32 * q;
                    v[u][q] = (i < nv && rq < r1) ? __ldg(V + (size_t)i * ld + rq) : TV(0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < RB; ++q) acc[u] += (TA)v[u][q] * wr[q];
        }
        store_slot_partials<NV>(acc, nv, out);
    }
}

// pass 1 (float64 modes): partial dots V^T w
template <int NV>
__global__ void __launch_bounds__(KT, 2) mdot_kernel(const double *__restrict__ V, int64_t ld, int nv,
                                                  const double *__restrict__ w, int64_t n,
                                                  double *__restrict__ partials, const FgState *fg) {
    pdl_trigger();
    pdl_wait();
    if (fg) nv = min(fg->k + 1, NV);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    stream_dots<NV, double, double>(V, ld, nv, w, r0, r1, partials + (size_t)blockIdx.x * KMAX);
}

// First Gram-Schmidt pass of the mixed modes: h1 = V^T w from the float32
// copy of the basis and w rounded to float32, float32 products and sums.
// The second pass (float64) removes whatever this pass leaves, so h = h1 + h2
// and the new basis vector keep float64 accuracy; the float32 pipe and the
// halved basis bytes replace the float64 multiply-adds of a full pass.
template <int NV>
__global__ void __launch_bounds__(KT, 4) mdot32_kernel(const float *__restrict__ V, int64_t ld, int nv,
                                                    const double *__restrict__ w, int64_t n,
                                                    double *__restrict__ partials, const FgState *fg) {
    pdl_trigger();
    pdl_wait();
    if (fg) nv = min(fg->k + 1, NV);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    stream_dots<NV, float, float>(V, ld, nv, w, r0, r1, partials + (size_t)blockIdx.x * KMAX);
}

// pass 2: w -= V h and partial dots V^T w (norm_only = 0);
// pass 3: w -= V h and partial ||w||^2   (norm_only = 1).
// With V32 (mixed modes) the dots of pass 2 are float32, from the float32
// copy of the basis and w rounded to float32: they only measure the small
// residue the first pass left, so their rounding leaves the basis orthogonal
// to ~1e-6 instead of 1e-15, while both updates stay float64 and keep the
// Arnoldi relation A Z = V H exact; half of the float64 multiply-adds of
// the pass go to the float32 pipe.
// NV <= 8: one thread per row does both.  Otherwise a thread first updates its row of the tile (the sum V[r, :] h in four
// independent chains, then one subtraction), writes it back and into shared
// memory; the warps then form the dots of the updated tile.  The basis tile
// is read from HBM in the update and again, from L1/L2, in the dots.
template <int NV>
__global__ void __launch_bounds__(KT, 2) update_dot_kernel(double *__restrict__ w, const double *__restrict__ V,
                                                        int64_t ld, int nv, const double *__restrict__ h,
                                                        int64_t n, double *__restrict__ partials, int norm_only,
                                                        const FgState *fg, const float *__restrict__ V32) {
    pdl_trigger();
    pdl_wait();
    if (fg) nv = min(fg->k + 1, NV);
    __shared__ double hs[KMAX];
    __shared__ double ws[KT];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    double nrm = 0.0;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    if constexpr (NV <= 8) {
        double acc[NV];
        float accf[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            acc[i] = 0.0;
            accf[i] = 0.f;
        }
        for (int64_t r = r0 + threadIdx.x; r < r1; r += KT) {
            double v[NV];
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i < nv) {
                    v[i] = __ldg(V + (size_t)i * ld + r);
                    s += v[i] * hs[i];
                }
            const double wr = w[r] - s;
            w[r] = wr;
            if (norm_only) {
                nrm += wr * wr;
            } else if (V32) {
                const float wf = (float)wr;
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    if (i < nv) accf[i] = fmaf(__ldg(V32 + (size_t)i * ld + r), wf, accf[i]);
            } else {
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    if (i < nv) acc[i] += v[i] * wr;
            }
        }
        if (V32 && !norm_only)
#pragma unroll
            for (int i = 0; i < NV; ++i) acc[i] = (double)accf[i];
        if (norm_only) store_cta_sum(nrm, partials + (size_t)blockIdx.x * KMAX);
        else store_row_partials<NV>(acc, nv, partials + (size_t)blockIdx.x * KMAX);
        return;
    }
    double acc[Slots<NV>::U];
    float accf[Slots<NV>::U];
    __shared__ float wsf[KT];
#pragma unroll
    for (int u = 0; u < Slots<NV>::U; ++u) {
        acc[u] = 0.0;
        accf[u] = 0.f;
    }
    for (int64_t t0 = r0; t0 < r1; t0 += KT) {
        const int64_t r = t0 + threadIdx.x;
        double wr = 0.0;
        if (r < r1) {
            double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i < nv) s[i & 3] += __ldg(V + (size_t)i * ld + r) * hs[i];
            wr = w[r] - ((s[0] + s[1]) + (s[2] + s[3]));
            w[r] = wr;
        }
        if (norm_only) {
            nrm += wr * wr;
        } else if (V32) {
            wsf[threadIdx.x] = (float)wr;
            __syncthreads();
            tile_dots<NV>(V32, ld, nv, t0, r1, wsf, accf);
            __syncthreads();
        } else {
            ws[threadIdx.x] = wr;
            __syncthreads();
            tile_dots<NV>(V, ld, nv, t0, r1, ws, acc);
            __syncthreads();
        }
    }
    if (norm_only) store_cta_sum(nrm, partials + (size_t)blockIdx.x * KMAX);
    else if (V32) store_slot_partials<NV>(accf, nv, partials + (size_t)blockIdx.x * KMAX);
    else store_slot_partials<NV>(acc, nv, partials + (size_t)blockIdx.x * KMAX);
}

// one warp per vector: lanes stride over the per-CTA partials in a fixed
// order, then a fixed shuffle tree (deterministic)
__global__ void reduce_partials_kernel(const double *__restrict__ partials, int nblocks, int nv,
                                       double *__restrict__ out, int accumulate, const FgState *fg) {
    pdl_trigger();
    pdl_wait();
    if (fg) nv = min(fg->k + 1, KMAX);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    for (int i = warp; i < nv; i += nw) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += partials[(size_t)b * KMAX + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = accumulate ? out[i] + s : s;
    }
}

// Column j of the Hessenberg matrix H (ld = restart + 1): h = h1 + h2 from
// the two Gram-Schmidt passes, h_{j+1,j} = sqrt(hn2).  Applies the previous
// rotations, forms rotation j, updates g.  scal[0] = |g_{j+1}| (estimate),
// scal[1] = h_{j+1,j}, scal[2] = ||A z_j|| (= sqrt(|h|^2 + h_{j+1,j}^2)),
// scal[3] = 1 on breakdown-free column, 0 if both entries of the rotation
// vanish; scal[4] non-finite flag.
//
// With a control block (device-side loop) j = fg->k, and the step's end
// test runs here: fg->its and fg->k advance, and the loop's condition is
// cleared when the estimate reaches rtol ||b||, on a (lucky) breakdown
// h_{j+1,j} <= 1e-14 ||A z_j||, at max_iters, at the restart length, or on
// a non-finite value (fg->flags bit 0).
__global__ void givens_kernel(double *H, int ld, int j, const double *h1, const double *h2,
                              const double *hn2, double *cs, double *sn, double *g, double *scal,
                              FgState *fg, cudaGraphConditionalHandle loop) {
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (fg) j = fg->k;
    double *col = H + (size_t)j * ld;
    double ss = 0.0;
    for (int i = 0; i <= j; ++i) {
        col[i] = h1[i] + h2[i];
        ss += col[i] * col[i];
    }
    const double hn = sqrt(fmax(hn2[0], 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    double c = 1.0, s = 0.0;
    if (den > 0.0) {
        c = col[j] / den;
        s = col[j + 1] / den;
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    scal[0] = fabs(g[j + 1]);
    scal[1] = hn;
    scal[2] = sqrt(ss + hn * hn);
    scal[3] = den > 0.0 ? 1.0 : 0.0;
    scal[4] = (isfinite(scal[0]) && isfinite(hn) && isfinite(den)) ? 0.0 : 1.0;
    if (fg) {
        const int its = fg->its + 1, k = j + 1;
        fg->its = its;
        fg->k = k;
        const bool bad = scal[4] != 0.0;
        if (bad) fg->flags |= 1;
        const bool stop = bad || scal[0] <= fg->rtol * fg->bnorm || hn <= 1e-14 * scal[2] ||
                          its >= fg->max_iters || k >= fg->m;
        cudaGraphSetConditional(loop, stop ? 0u : 1u);
    }
}

// v = w / scal[idx]; with a control block v is column fg->k of the basis
// whose first column is v (leading dimension ld)
__global__ void scale_copy_kernel(const double *__restrict__ w, double *__restrict__ v, float *__restrict__ v32,
                                  const double *__restrict__ scal, int idx, int64_t n, const FgState *fg,
                                  int64_t ld) {
    pdl_trigger();
    pdl_wait();
    if (fg) {
        v += (size_t)fg->k * ld;
        if (v32) v32 += (size_t)fg->k * ld;
    }
    const double inv = 1.0 / scal[idx];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double a = w[r] * inv;
        v[r] = a;
        if (v32) v32[r] = (float)a;
    }
}

// start of a cycle: beta = sqrt(nrm2), v0 = r / beta, g = (beta, 0, ...)
// (device-side loop: also k = 0 and the inner loop's condition set)
__global__ void init_basis_kernel(const double *__restrict__ r, double *__restrict__ v0, float *__restrict__ v0f,
                                  double *__restrict__ g, int m, const double *__restrict__ nrm2, int64_t n,
                                  FgState *fg, cudaGraphConditionalHandle loop) {
    if (fg && blockIdx.x == 0 && threadIdx.x == 0) {
        fg->k = 0;
        cudaGraphSetConditional(loop, 1u);
    }
    const double beta = sqrt(nrm2[0]);
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = r[i] * inv;
        v0[i] = a;
        if (v0f) v0f[i] = (float)a;
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta : 0.0;
}

// y = H(1:k,1:k)^{-1} g(1:k), upper triangular
__global__ void backsolve_kernel(const double *H, int ld, int k, const double *g, double *y, const FgState *fg) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (fg) k = fg->k;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= H[(size_t)j * ld + i] * y[j];
        y[i] = s / H[(size_t)i * ld + i];
    }
}

template <class T>
__global__ void combine_kernel(double *__restrict__ x, const T *__restrict__ Z, int64_t ld, int k,
                               const double *__restrict__ y, int64_t n, const FgState *fg) {
    if (fg) k = min(fg->k, KMAX);
    __shared__ double ys[KMAX];
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = x[r];
        for (int i = 0; i < k; ++i) s += (double)Z[(size_t)i * ld + r] * ys[i];
        x[r] = s;
    }
}

template <class TI, class TO>
__global__ void take_column_kernel(const TI *__restrict__ V, int64_t ld, const FgState *fg, TO *__restrict__ dst,
                                   int64_t n, cudaGraphConditionalHandle sel, TO *__restrict__ zero) {
    pdl_trigger();
    if (sel && blockIdx.x == 0 && threadIdx.x == 0) {
        const int nv = fg->k + 1;
        int c = 0;
        while (c < NV_CLASSES - 1 && nv > nv_class_bound(c)) ++c;
        cudaGraphSetConditional(sel, (unsigned)c);
    }
    const TI *v = V + (size_t)fg->k * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        dst[i] = (TO)v[i];
        if (zero) zero[i] = TO(0);
    }
}

template <class T>
__global__ void store_column_kernel(const T *__restrict__ z, double *__restrict__ zfix, double *__restrict__ Z,
                                    int64_t ld, const FgState *fg, int64_t n) {
    pdl_trigger();
    pdl_wait();
    double *zc = Z + (size_t)fg->k * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)z[i];
        zfix[i] = v;
        zc[i] = v;
    }
}

// start of a device-driven solve: ||b|| and ||r0|| from the squared norms,
// run the outer loop while the residual is above rtol ||b||
__global__ void fg_start_kernel(const double *scal, FgState *fg, cudaGraphConditionalHandle outer) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double bn = sqrt(scal[5]), beta = sqrt(scal[6]);
    fg->bnorm = bn;
    fg->beta = beta;
    fg->r0 = beta;
    fg->its = 0;
    fg->cycles = 0;
    fg->k = 0;
    fg->flags = (isfinite(bn) && isfinite(beta)) ? 0 : 1;
    const bool go = fg->flags == 0 && bn > 0.0 && beta > fg->rtol * bn && fg->max_iters > 0;
    cudaGraphSetConditional(outer, go ? 1u : 0u);
}

// end of a cycle: the new true residual decides whether to restart
__global__ void fg_cycle_kernel(const double *scal, FgState *fg, cudaGraphConditionalHandle outer) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double beta = sqrt(scal[6]);
    fg->beta = beta;
    fg->cycles += 1;
    if (!isfinite(beta)) fg->flags |= 1;
    const bool go = fg->flags == 0 && beta > fg->rtol * fg->bnorm && fg->its < fg->max_iters;
    cudaGraphSetConditional(outer, go ? 1u : 0u);
}

inline int egrid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

// Float64 FMA throughput of this GPU (measurement support for the roofline
// of the float64-bound kernels): 8 independent FMA chains per thread, one
// store per thread so that nothing is optimised away.
__global__ void __launch_bounds__(256) fp64_rate_kernel(double *out, double a, double b, int iters) {
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

fsi_status measure_fp64_rate(int num_sms, cudaStream_t s, double *gflops) {
    const int blocks = num_sms * 8, threads = 256, iters = 2048;
    DevBuf out;
    FSI_TRY(out.alloc((size_t)blocks * threads * 8));
    cudaEvent_t e0, e1;
    FSI_CUDA(cudaEventCreate(&e0));
    FSI_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        FSI_CUDA(cudaEventRecord(e0, s));
        fp64_rate_kernel<<<blocks, threads, 0, s>>>(out.as<double>(), 0.999999, 1e-7, iters);
        FSI_CUDA(cudaEventRecord(e1, s));
        FSI_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        FSI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);     // first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gflops = 2.0 * (double)blocks * threads * iters * 8 / (best * 1e-3) / 1e9;
    return FSI_OK;
}

#define FSI_NV_SWITCH(nv, CALL)                          \
    do {                                                 \
        if ((nv) <= 1) { CALL(1); }                      \
        else if ((nv) <= 2) { CALL(2); }                 \
        else if ((nv) <= 4) { CALL(4); }                 \
        else if ((nv) <= 8) { CALL(8); }                 \
        else if ((nv) <= 16) { CALL(16); }               \
        else if ((nv) <= 32) { CALL(32); }               \
        else { CALL(KMAX); }                             \
    } while (0)

fsi_status launch_mdot(const double *V, int64_t ld, int nv, const double *w, int64_t n,
                       double *partials, int nblocks, cudaStream_t s, const FgState *fg) {
    if (nv > KMAX) { set_error("too many Krylov vectors"); return FSI_ERR_ARG; }
#define CALL_MDOT(NV) FSI_CUDA(launch_pdl(mdot_kernel<NV>, dim3(nblocks), dim3(KT), 0, s, V, ld, nv, w, n, partials, fg))
    FSI_NV_SWITCH(nv, CALL_MDOT);
#undef CALL_MDOT
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_mdot32(const float *V, int64_t ld, int nv, const double *w, int64_t n, double *partials,
                         int nblocks, cudaStream_t s, const FgState *fg) {
    if (nv > KMAX) { set_error("too many Krylov vectors"); return FSI_ERR_ARG; }
#define CALL_MDOT32(NV) FSI_CUDA(launch_pdl(mdot32_kernel<NV>, dim3(nblocks), dim3(KT), 0, s, V, ld, nv, w, n, partials, fg))
    FSI_NV_SWITCH(nv, CALL_MDOT32);
#undef CALL_MDOT32
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_update_dot(double *w, const double *V, int64_t ld, int nv, const double *h,
                             int64_t n, double *partials, int nblocks, int norm_only, cudaStream_t s,
                             const FgState *fg, const float *V32) {
    if (nv > KMAX) { set_error("too many Krylov vectors"); return FSI_ERR_ARG; }
#define CALL_UPD(NV) FSI_CUDA(launch_pdl(update_dot_kernel<NV>, dim3(nblocks), dim3(KT), 0, s, w, V, ld, nv, h, n, partials, norm_only, fg, V32))
    FSI_NV_SWITCH(nv, CALL_UPD);
#undef CALL_UPD
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_reduce_partials(const double *partials, int nblocks, int nv, double *out, int accumulate,
                                  cudaStream_t s, const FgState *fg) {
    FSI_CUDA(launch_pdl(reduce_partials_kernel, dim3(1), dim3(1024), 0, s, partials, nblocks, nv, out, accumulate, fg));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_givens(double *H, int ld, int j, const double *h1, const double *h2, const double *hn2,
                         double *cs, double *sn, double *g, double *scal, cudaStream_t s, FgState *fg,
                         cudaGraphConditionalHandle loop) {
    FSI_CUDA(launch_pdl(givens_kernel, dim3(1), dim3(32), 0, s, H, ld, j, h1, h2, hn2, cs, sn, g, scal, fg, loop));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_scale_copy(const double *w, double *v, const double *scal, int idx, int64_t n,
                             cudaStream_t s, const FgState *fg, int64_t ld, float *v32) {
    FSI_CUDA(launch_pdl(scale_copy_kernel, dim3(egrid(n)), dim3(256), 0, s, w, v, v32, scal, idx, n, fg, ld));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_init_basis(const double *r, double *v0, double *g, int m, const double *nrm2, int64_t n,
                             cudaStream_t s, FgState *fg, cudaGraphConditionalHandle loop, float *v0f) {
    init_basis_kernel<<<egrid(n), 256, 0, s>>>(r, v0, v0f, g, m, nrm2, n, fg, loop);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_backsolve(const double *H, int ld, int k, const double *g, double *y, cudaStream_t s,
                            const FgState *fg) {
    backsolve_kernel<<<1, 32, 0, s>>>(H, ld, k, g, y, fg);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

template <class T>
fsi_status launch_combine(double *x, const T *Z, int64_t ld, int k, const double *y, int64_t n,
                          cudaStream_t s, const FgState *fg) {
    combine_kernel<T><<<egrid(n), 256, 0, s>>>(x, Z, ld, k, y, n, fg);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

template fsi_status launch_combine<float>(double *, const float *, int64_t, int, const double *, int64_t,
                                          cudaStream_t, const FgState *);
template fsi_status launch_combine<double>(double *, const double *, int64_t, int, const double *, int64_t,
                                           cudaStream_t, const FgState *);

template <class TI, class TO>
fsi_status launch_take_column(const TI *V, int64_t ld, const FgState *fg, TO *dst, int64_t n, cudaStream_t s,
                              cudaGraphConditionalHandle sel, TO *zero) {
    take_column_kernel<TI, TO><<<egrid(n), 256, 0, s>>>(V, ld, fg, dst, n, sel, zero);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
template fsi_status launch_take_column<double, float>(const double *, int64_t, const FgState *, float *, int64_t,
                                                      cudaStream_t, cudaGraphConditionalHandle, float *);
template fsi_status launch_take_column<double, double>(const double *, int64_t, const FgState *, double *, int64_t,
                                                       cudaStream_t, cudaGraphConditionalHandle, double *);

template <class T>
fsi_status launch_store_column(const T *z, double *zfix, double *Z, int64_t ld, const FgState *fg, int64_t n,
                               cudaStream_t s) {
    FSI_CUDA(launch_pdl(store_column_kernel<T>, dim3(egrid(n)), dim3(256), 0, s, z, zfix, Z, ld, fg, n));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
template fsi_status launch_store_column<float>(const float *, double *, double *, int64_t, const FgState *, int64_t,
                                               cudaStream_t);
template fsi_status launch_store_column<double>(const double *, double *, double *, int64_t, const FgState *,
                                                int64_t, cudaStream_t);

fsi_status launch_fg_start(const double *scal, FgState *fg, cudaGraphConditionalHandle outer, cudaStream_t s) {
    fg_start_kernel<<<1, 32, 0, s>>>(scal, fg, outer);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_fg_cycle(const double *scal, FgState *fg, cudaGraphConditionalHandle outer, cudaStream_t s) {
    fg_cycle_kernel<<<1, 32, 0, s>>>(scal, fg, outer);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

}  // namespace fsi
