// Sparse matrix-vector products: level residuals r = b - A x, the outer
// float64 product w = A z, restriction b_c = R r and prolongation x += P e.
//
// Operators on the solve path are streamed from a length-binned ELL copy
// (ell_spmv_kernel): one thread per row, 32 rows of equal length per warp,
// every (column, value) load a full coalesced line and independent of the
// others, no row pointers and no cross-lane reduction.  Row lengths of the
// Q2/Q1 operators vary from 1 to ~110 with the node type (vertex, edge,
// interior; K, S, F, A, V, W rows), which is what a fixed number of lanes
// per row handles badly.  The CSR kernel below serves values without an ELL
// copy (e.g. dA/dmu_s on the fine pattern).
//
// CSR kernel: G threads cooperate on one row (G = 4..32 picked from the mean row length
// at set-up) so that the value and column streams are read in contiguous,
// coalesced runs; the partial sums are combined with warp shuffles.  Values
// and columns are streamed once (read-only, no L1 allocation); the gathered
// vector x stays in L2.  Accumulation is in the wider of the matrix and
// vector precisions.
#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "context.h"

namespace fsi {

namespace {

template <class TA, class TX> struct Acc { using type = float; };
template <class TX> struct Acc<double, TX> { using type = double; };
template <> struct Acc<float, double> { using type = double; };

// G lanes per row, 32/G rows per warp at a time; each lane issues U
// independent (column, value) loads and then U gathers before using them, so
// a warp keeps 32*U loads in flight instead of one dependent chain per row.
template <int G, int U, class TA, class TX, class TY>
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, const int32_t *__restrict__ ptr,
                                                   const int32_t *__restrict__ col,
                                                   const TA *__restrict__ val, const TX *__restrict__ x,
                                                   const TY *__restrict__ b, TY *__restrict__ y, int mode,
                                                   TY *__restrict__ zero_out) {
    using AT = typename Acc<TA, TX>::type;
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x % G;
    const int64_t rows_per_grid = ((int64_t)gridDim.x * blockDim.x) / G;
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    while (true) {
        // lane 0 holds the warp's smallest row: a warp-uniform exit test keeps
        // every lane present for the shuffles below
        const int64_t first = __shfl_sync(0xffffffffu, row, 0);
        if (first >= n) break;
        const bool active = row < n;
        AT acc = 0;
        if (active) {
            const int k0 = __ldg(ptr + row), k1 = __ldg(ptr + row + 1);
            for (int k = k0 + lane; k < k1; k += G * U) {
                int c[U];
                TA v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int kk = k + u * G;
                    c[u] = kk < k1 ? __ldcs(col + kk) : -1;
                    v[u] = kk < k1 ? __ldcs(val + kk) : TA(0);
                }
                TX xv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : TX(0);
#pragma unroll
                for (int u = 0; u < U; ++u) acc += (AT)v[u] * (AT)xv[u];
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
        if (active && lane == 0) {
            if (mode == SPMV_SET) y[row] = (TY)acc;
            else if (mode == SPMV_RESID) y[row] = (TY)((AT)b[row] - acc);
            else y[row] = (TY)((AT)y[row] + acc);
            if (zero_out) zero_out[row] = TY(0);
        }
        row += rows_per_grid;
    }
}

template <int G, int U, class TA, class TX, class TY>
fsi_status run(const DevCSR &A, const TA *val, const TX *x, const TY *b, TY *y, int mode, cudaStream_t s,
               TY *zero_out) {
    const int threads = 256;
    int64_t blocks = (A.n_rows * G + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    FSI_CUDA(launch_pdl(spmv_kernel<G, U, TA, TX, TY>, dim3((unsigned)blocks), dim3(threads), 0, s, A.n_rows,
                        A.ptr.as<int32_t>(), A.col.as<int32_t>(), val, x, b, y, mode, zero_out));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

// ---- binned ELL ----------------------------------------------------------
// Warp = one slab of 32/G rows of one bin; G lanes per row, lane `sub` of a
// row takes entries sub, sub + G, ...  Per pass a lane issues UNR
// predicated (column, value) loads, all independent, then their gathers, so
// a row of length len costs ceil(len / (G UNR)) dependent load-gather steps:
// G = 1 on large operators (no shuffles; enough rows to hide latency), up to
// 16 on small ones (few rows, short chains).  STREAM: evict-first loads for
// operators larger than L2 is useful for; small ones stay cached.
// float32 with one lane per row: <= 40 registers, 6 CTAs (48 warps) per SM
template <int G, bool STREAM, int UNR, class TA, class TX, class TY>
__global__ void __launch_bounds__(256, (G == 1 && sizeof(TA) == 4) ? 6 : 0) ell_spmv_kernel(const EllBin *__restrict__ bins, int nbins, int64_t nslabs,
                                                       const int32_t *__restrict__ perm,
                                                       const int32_t *__restrict__ col,
                                                       const TA *__restrict__ val, const TX *__restrict__ x,
                                                       const TY *__restrict__ b, TY *__restrict__ y, int mode,
                                                       TY *__restrict__ zero_out) {
    using AT = typename Acc<TA, TX>::type;
    pdl_trigger();
    const int64_t slab = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (slab >= nslabs) return;                      // whole warps
    const int lane = threadIdx.x % 32, sub = lane % G;
    int lo = 0, hi = nbins - 1;                      // last bin with slab0 <= slab
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (__ldg(&bins[mid].slab0) <= slab) lo = mid;
        else hi = mid - 1;
    }
    const int64_t off = __ldg(&bins[lo].off);
    const int rows = __ldg(&bins[lo].rows), len = __ldg(&bins[lo].len), stride = __ldg(&bins[lo].stride);
    const int first = __ldg(&bins[lo].first), slab0 = __ldg(&bins[lo].slab0);
    const int t = (int)(slab - slab0) * (32 / G) + lane / G;   // < stride
    const int32_t *cp = col + off + t;
    const TA *vp = val + off + t;
    pdl_wait();                                      // x, b, y belong to earlier kernels
    AT a0 = 0, a1 = 0;
    if constexpr (G == 1) {
        // large operators: full chunks, then the remainder one by one
        int k = 0;
        for (; k + UNR <= len; k += UNR) {
            int c[UNR];
            TA v[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                c[u] = STREAM ? __ldcs(cp + (int64_t)(k + u) * stride) : __ldg(cp + (int64_t)(k + u) * stride);
                v[u] = STREAM ? __ldcs(vp + (int64_t)(k + u) * stride) : __ldg(vp + (int64_t)(k + u) * stride);
            }
            TX xv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) xv[u] = __ldg(x + c[u]);
#pragma unroll
            for (int u = 0; u < UNR; u += 2) {
                a0 += (AT)v[u] * (AT)xv[u];
                if (u + 1 < UNR) a1 += (AT)v[u + 1] * (AT)xv[u + 1];
            }
        }
        for (; k < len; ++k) {
            const int c = STREAM ? __ldcs(cp + (int64_t)k * stride) : __ldg(cp + (int64_t)k * stride);
            const TA v = STREAM ? __ldcs(vp + (int64_t)k * stride) : __ldg(vp + (int64_t)k * stride);
            a0 += (AT)v * (AT)__ldg(x + c);
        }
    } else {
        for (int k = sub; k < len; k += G * UNR) {
            int c[UNR];
            TA v[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int kk = k + G * u;
                const int64_t q = (int64_t)kk * stride;
                if (kk < len) {
                    c[u] = STREAM ? __ldcs(cp + q) : __ldg(cp + q);
                    v[u] = STREAM ? __ldcs(vp + q) : __ldg(vp + q);
                } else {
                    c[u] = 0;
                    v[u] = TA(0);
                }
            }
            TX xv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) xv[u] = __ldg(x + c[u]);
#pragma unroll
            for (int u = 0; u < UNR; u += 2) {
                a0 += (AT)v[u] * (AT)xv[u];
                if (u + 1 < UNR) a1 += (AT)v[u + 1] * (AT)xv[u + 1];
            }
        }
    }
    AT acc = a0 + a1;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    if (sub == 0 && t < rows) {
        const int64_t r = __ldg(perm + first + t);
        if (mode == SPMV_SET) y[r] = (TY)acc;
        else if (mode == SPMV_RESID) y[r] = (TY)((AT)b[r] - acc);
        else y[r] = (TY)((AT)y[r] + acc);
        if (zero_out) zero_out[r] = TY(0);
    }
}

template <int G, bool STREAM, class TA, class TX, class TY>
fsi_status run_ell_g(const DevEll &E, const TA *val, const TX *x, const TY *b, TY *y, int mode, cudaStream_t s,
                     TY *zero_out) {
    const int threads = 256;
    const int64_t blocks = (E.nslabs * 32 + threads - 1) / threads;
    if (blocks < 1) return FSI_OK;
    constexpr int UNR = sizeof(TA) == 8 ? 6 : 8;
    FSI_CUDA(launch_pdl(ell_spmv_kernel<G, STREAM, UNR, TA, TX, TY>, dim3((unsigned)blocks), dim3(threads), 0, s,
                        E.bins.as<EllBin>(), E.nbins, E.nslabs, E.perm.as<int32_t>(), E.col.as<int32_t>(), val, x,
                        b, y, mode, zero_out));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

// The kernel's lanes per row must equal the layout's: a bin's slabs hold
// 32 / G rows, so any other G maps slabs to rows past the bin.
template <bool STREAM, class TA, class TX, class TY>
fsi_status run_ell_s(const DevEll &E, const TA *val, const TX *x, const TY *b, TY *y, int mode, cudaStream_t s,
                     TY *z) {
    switch (E.G) {
        case 1: return run_ell_g<1, STREAM>(E, val, x, b, y, mode, s, z);
        case 4: return run_ell_g<4, STREAM>(E, val, x, b, y, mode, s, z);
        case 8: return run_ell_g<8, STREAM>(E, val, x, b, y, mode, s, z);
        case 16: return run_ell_g<16, STREAM>(E, val, x, b, y, mode, s, z);
        default: set_error("ELL copy with an unsupported lane count"); return FSI_ERR_STATE;
    }
}

template <class TA, class TX, class TY>
fsi_status run_ell(const DevEll &E, const TA *val, const TX *x, const TY *b, TY *y, int mode, cudaStream_t s,
                   TY *z) {
    return E.stream ? run_ell_s<true>(E, val, x, b, y, mode, s, z) : run_ell_s<false>(E, val, x, b, y, mode, s, z);
}

template <class T>
__global__ void zero_kernel(T *__restrict__ v, int64_t n) {
    pdl_trigger();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = T(0);
}

// one thread per CSR row: copy its entries to their ELL positions
template <class T>
__global__ void ell_fill_kernel(int64_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                const T *__restrict__ val, const int64_t *__restrict__ base,
                                const int32_t *__restrict__ rstride, int32_t *__restrict__ ecol,
                                T *__restrict__ eval) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int k0 = ptr[r], k1 = ptr[r + 1];
        const int64_t b0 = base[r], st = rstride[r];
        for (int k = k0; k < k1; ++k) {
            const int64_t q = b0 + (int64_t)(k - k0) * st;
            if (ecol) ecol[q] = col[k];
            eval[q] = val[k];
        }
    }
}

// one thread per stored row of a row-subset copy: row rows[i] of the CSR,
// entries whose column has keep[col] != 0, to positions base[i] + m stride[i]
template <class T>
__global__ void ell_fill_subset_kernel(int64_t nsub, const int32_t *__restrict__ rows,
                                       const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                       const T *__restrict__ val, const uint8_t *__restrict__ keep,
                                       const int64_t *__restrict__ base, const int32_t *__restrict__ rstride,
                                       int32_t *__restrict__ ecol, T *__restrict__ eval) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsub; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rows[i];
        const int64_t b0 = base[i], st = rstride[i];
        int64_t m = 0;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) {
            const int32_t c = col[k];
            if (!keep[c]) continue;
            const int64_t q = b0 + m * st;
            if (ecol) ecol[q] = c;
            eval[q] = val[k];
            ++m;
        }
    }
}

// x += a y, then y = 0 (the multiplicative sweep's correction is consumed)
template <class T>
__global__ void axpy_clear_kernel(T *__restrict__ x, T *__restrict__ y, T a, int64_t n) {
    pdl_trigger();
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * y[i];
        y[i] = T(0);
    }
}

}  // namespace

// Host: bins from the row lengths, then the fill kernel copies columns and
// values.  The per-row ELL bases are kept only for the fill (freed here).
fsi_status build_ell(DevCSR &A, cudaStream_t s, bool concurrent, int force_G) {
    DevEll &E = A.ell;
    const int64_t n = A.n_rows;
    if (n == 0 || A.nnz == 0 || !A.val64.p) return FSI_OK;
    if (n > INT32_MAX) { set_error("ELL copy: too many rows"); return FSI_ERR_ARG; }
    std::vector<int32_t> p32(n + 1);
    FSI_CUDA(cudaMemcpyAsync(p32.data(), A.ptr.p, (n + 1) * 4, cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    // longest rows first: the slabs that run longest are scheduled first and
    // the short ones fill in behind them (no long tail at the end of the grid)
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return p32[a + 1] - p32[a] > p32[b + 1] - p32[b]; });
    // lanes per row.  One lane per row issues the least work and serves
    // large operators (>= 150k rows: several waves of warps) and operators of
    // a batch (the problems' launches run side by side).  A small operator
    // alone on the GPU is latency-bound: its few rows get G lanes each
    // (rows x G >= 3e5 threads, G <= 16) so that a row of ~110 entries is one
    // or two dependent load-gather steps instead of fourteen.  Measured per
    // launch on the 256^2 hierarchy: 32^2 level 21 -> 7 us (G = 16); at
    // 128^2, G = 2 was slower than G = 1 (43 vs 32 us).
    int G = 1;
    if (!concurrent && n < 150000)
        while (G < 16 && n * G < 300000) G *= 2;
    if (G == 2) G = 4;
    if (force_G == 1 || force_G == 4 || force_G == 8 || force_G == 16) G = force_G;   // layout autotuner
    E.G = G;
    E.stream = (double)A.nnz * 12.0 > 64e6;
    std::vector<EllBin> bins;
    std::vector<int64_t> base(n);
    std::vector<int32_t> rstride(n);
    int64_t off = 0, slabs = 0;
    for (int64_t i = 0; i < n;) {
        const int len = p32[order[i] + 1] - p32[order[i]];
        int64_t j = i;
        while (j < n && p32[order[j] + 1] - p32[order[j]] == len) ++j;
        EllBin B{};
        B.off = off;
        B.rows = (int32_t)(j - i);
        B.len = len;
        const int64_t rps = 32 / G;               // rows per slab
        B.stride = (int32_t)((B.rows + rps - 1) / rps * rps);
        B.first = (int32_t)i;
        B.slab0 = (int32_t)slabs;
        for (int64_t t = i; t < j; ++t) {
            base[order[t]] = off + (t - i);
            rstride[order[t]] = B.stride;
        }
        bins.push_back(B);
        off += (int64_t)B.stride * len;
        slabs += (int64_t)B.stride * G / 32;
        i = j;
    }
    if (slabs > INT32_MAX) { set_error("ELL copy: too many slabs"); return FSI_ERR_ARG; }
    E.nbins = (int)bins.size();
    E.nslabs = slabs;
    E.size = off;
    FSI_TRY(E.bins.alloc(bins.size() * sizeof(EllBin)));
    FSI_CUDA(cudaMemcpyAsync(E.bins.p, bins.data(), bins.size() * sizeof(EllBin), cudaMemcpyHostToDevice, s));
    FSI_TRY(E.perm.alloc((size_t)n * 4));
    FSI_CUDA(cudaMemcpyAsync(E.perm.p, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    DevBuf dbase, dstride;
    FSI_TRY(dbase.alloc((size_t)n * 8));
    FSI_TRY(dstride.alloc((size_t)n * 4));
    FSI_CUDA(cudaMemcpyAsync(dbase.p, base.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(dstride.p, rstride.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    FSI_TRY(E.col.alloc((size_t)E.size * 4));
    FSI_TRY(E.val64.alloc((size_t)E.size * 8));
    FSI_CUDA(cudaMemsetAsync(E.col.p, 0, (size_t)E.size * 4, s));
    FSI_CUDA(cudaMemsetAsync(E.val64.p, 0, (size_t)E.size * 8, s));
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    ell_fill_kernel<double><<<(unsigned)g, 256, 0, s>>>(n, A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                         A.val64.as<double>(), dbase.as<int64_t>(),
                                                         dstride.as<int32_t>(), E.col.as<int32_t>(),
                                                         E.val64.as<double>());
    count_launch();
    FSI_CUDA(cudaGetLastError());
    if (A.val32.p) {
        FSI_TRY(E.val32.alloc((size_t)E.size * 4));
        FSI_CUDA(cudaMemsetAsync(E.val32.p, 0, (size_t)E.size * 4, s));
        ell_fill_kernel<float><<<(unsigned)g, 256, 0, s>>>(n, A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                            A.val32.as<float>(), dbase.as<int64_t>(),
                                                            dstride.as<int32_t>(), nullptr, E.val32.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    E.fbase = std::move(dbase);           // kept: refills after the CSR values change
    E.fstride = std::move(dstride);
    FSI_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    return FSI_OK;
}

// new CSR values, same pattern: re-fill the ELL copy's float64 values (and
// its float32 values when both float32 copies exist) through the fill map
fsi_status ell_refill(DevCSR &A, cudaStream_t s) {
    DevEll &E = A.ell;
    if (E.nbins == 0) return FSI_OK;
    if (!E.fbase.p) { set_error("ELL copy without a fill map"); return FSI_ERR_STATE; }
    const int64_t n = A.n_rows;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    ell_fill_kernel<double><<<(unsigned)g, 256, 0, s>>>(n, A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                         A.val64.as<double>(), E.fbase.as<int64_t>(),
                                                         E.fstride.as<int32_t>(), nullptr, E.val64.as<double>());
    count_launch();
    FSI_CUDA(cudaGetLastError());
    if (E.val32.p && A.val32.p) {
        ell_fill_kernel<float><<<(unsigned)g, 256, 0, s>>>(n, A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                            A.val32.as<float>(), E.fbase.as<int64_t>(),
                                                            E.fstride.as<int32_t>(), nullptr, E.val32.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    return FSI_OK;
}

// float32 values of an existing ELL copy from A.val32 (after make_f32)
fsi_status ell_fill_f32(DevCSR &A, cudaStream_t s) {
    DevEll &E = A.ell;
    if (E.nbins == 0 || E.val32.p || !A.val32.p) return FSI_OK;
    if (E.fbase.p) {
        FSI_TRY(E.val32.alloc((size_t)E.size * 4));
        FSI_CUDA(cudaMemsetAsync(E.val32.p, 0, (size_t)E.size * 4, s));
        return ell_refill(A, s);
    }
    // the ELL position of CSR entry k is recovered from the float64 copy's
    // layout: rebuild the per-row bases from the bins (host)
    const int64_t n = A.n_rows;
    std::vector<EllBin> bins(E.nbins);
    std::vector<int32_t> order(n);
    FSI_CUDA(cudaMemcpyAsync(bins.data(), E.bins.p, bins.size() * sizeof(EllBin), cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaMemcpyAsync(order.data(), E.perm.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> base(n);
    std::vector<int32_t> rstride(n);
    for (const EllBin &B : bins)
        for (int t = 0; t < B.rows; ++t) {
            base[order[B.first + t]] = B.off + t;
            rstride[order[B.first + t]] = B.stride;
        }
    DevBuf dbase, dstride;
    FSI_TRY(dbase.alloc((size_t)n * 8));
    FSI_TRY(dstride.alloc((size_t)n * 4));
    FSI_CUDA(cudaMemcpyAsync(dbase.p, base.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(dstride.p, rstride.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    FSI_TRY(E.val32.alloc((size_t)E.size * 4));
    FSI_CUDA(cudaMemsetAsync(E.val32.p, 0, (size_t)E.size * 4, s));
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    ell_fill_kernel<float><<<(unsigned)g, 256, 0, s>>>(n, A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                        A.val32.as<float>(), dbase.as<int64_t>(),
                                                        dstride.as<int32_t>(), nullptr, E.val32.as<float>());
    count_launch();
    FSI_CUDA(cudaGetLastError());
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

template <class TA, class TX, class TY>
fsi_status launch_spmv(const DevCSR &A, const TA *val, const TX *x, const TY *b, TY *y, int mode,
                       cudaStream_t s, TY *zero_out) {
    if (A.n_rows == 0) return FSI_OK;
    if (A.ell.nbins > 0) {
        const void *ev = nullptr;
        if ((const void *)val == A.val64.p) ev = A.ell.val64.p;
        else if ((const void *)val == A.val32.p) ev = A.ell.val32.p;
        if (ev) return run_ell<TA, TX, TY>(A.ell, static_cast<const TA *>(ev), x, b, y, mode, s, zero_out);
    }
    // float64 accumulation: at most 4 lanes per row, so the shuffle tree adds
    // 2 float64 steps per lane instead of 5 (float64 issue rate is the limit;
    // measured: 2 lanes per row are slower, 184 vs 168 us on the 256^2 level)
    const bool f64 = std::is_same<typename Acc<TA, TX>::type, double>::value;
    const int G = f64 ? (A.group >= 4 ? 4 : A.group) : A.group;
    // loads per lane and pass: enough to cover a mean-length row in one pass
    const double avg = A.n_rows ? (double)A.nnz / (double)A.n_rows : 0.0;
    const int need = (int)((avg + G - 1) / G);
    const int U = need <= 2 ? 2 : (need <= 4 ? 4 : (need <= 6 ? 6 : 8));
#define FSI_SPMV_U(GG)                                              \
    switch (U) {                                                    \
        case 2: return run<GG, 2>(A, val, x, b, y, mode, s, zero_out);  \
        case 4: return run<GG, 4>(A, val, x, b, y, mode, s, zero_out);  \
        case 6: return run<GG, 6>(A, val, x, b, y, mode, s, zero_out);  \
        default: return run<GG, 8>(A, val, x, b, y, mode, s, zero_out); \
    }
    switch (G) {
        case 1: FSI_SPMV_U(1);
        case 2: FSI_SPMV_U(2);
        case 4: FSI_SPMV_U(4);
        case 8: FSI_SPMV_U(8);
        default: FSI_SPMV_U(16);
    }
#undef FSI_SPMV_U
}

template fsi_status launch_spmv<double, double, double>(const DevCSR &, const double *, const double *,
                                                        const double *, double *, int, cudaStream_t, double *);
template fsi_status launch_spmv<float, float, float>(const DevCSR &, const float *, const float *,
                                                     const float *, float *, int, cudaStream_t, float *);

template <class T>
fsi_status launch_zero(T *v, int64_t n, cudaStream_t s) {
    if (n == 0) return FSI_OK;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    zero_kernel<T><<<(unsigned)g, 256, 0, s>>>(v, n);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
template fsi_status launch_zero<float>(float *, int64_t, cudaStream_t);
template fsi_status launch_zero<double>(double *, int64_t, cudaStream_t);

// Binned-ELL copy of a row subset of A restricted to the columns with
// keep[c] != 0: the rows keep their indices in A (perm holds them), so a
// product writes only those rows of its output.  Row lengths come from the
// host copy `pat` of A's pattern; columns and values are copied on the device
// from A's CSR.  Bins, lane count and streaming rule as in build_ell, taken
// on the subset's size.
fsi_status build_ell_subset(const DevCSR &A, const HostCSR &pat, const std::vector<int32_t> &rows,
                            const std::vector<uint8_t> &keep, const uint8_t *d_keep, DevEll &E,
                            cudaStream_t s, bool concurrent) {
    E = DevEll();
    const int64_t n = (int64_t)rows.size();
    if (n == 0) return FSI_OK;
    if ((int64_t)pat.ptr.size() != A.n_rows + 1 || (int64_t)keep.size() != A.n_cols) {
        set_error("ELL subset: pattern or column mask does not match the operator");
        return FSI_ERR_ARG;
    }
    std::vector<int32_t> len(n);
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t r = rows[i];
        if (r < 0 || r >= A.n_rows) { set_error("ELL subset: row out of range"); return FSI_ERR_ARG; }
        int c = 0;
        for (int64_t k = pat.ptr[r]; k < pat.ptr[r + 1]; ++k) c += keep[pat.col[k]] ? 1 : 0;
        len[i] = c;
        nnz += c;
    }
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len[a] > len[b]; });
    int G = 1;
    if (!concurrent && n < 150000)
        while (G < 16 && n * G < 300000) G *= 2;
    if (G == 2) G = 4;
    E.G = G;
    E.stream = (double)nnz * 12.0 > 64e6;
    std::vector<EllBin> bins;
    std::vector<int64_t> base(n);
    std::vector<int32_t> rstride(n), srows(n);
    int64_t off = 0, slabs = 0;
    for (int64_t i = 0; i < n;) {
        const int l = len[order[i]];
        int64_t j = i;
        while (j < n && len[order[j]] == l) ++j;
        EllBin B{};
        B.off = off;
        B.rows = (int32_t)(j - i);
        B.len = l;
        const int64_t rps = 32 / G;
        B.stride = (int32_t)((B.rows + rps - 1) / rps * rps);
        B.first = (int32_t)i;
        B.slab0 = (int32_t)slabs;
        for (int64_t t = i; t < j; ++t) {
            base[t] = off + (t - i);
            rstride[t] = B.stride;
            srows[t] = rows[order[t]];
        }
        bins.push_back(B);
        off += (int64_t)B.stride * l;
        slabs += (int64_t)B.stride * G / 32;
        i = j;
    }
    if (slabs > INT32_MAX) { set_error("ELL subset: too many slabs"); return FSI_ERR_ARG; }
    E.nbins = (int)bins.size();
    E.nslabs = slabs;
    E.size = off;
    E.nnz = nnz;
    FSI_TRY(E.bins.alloc(bins.size() * sizeof(EllBin)));
    FSI_CUDA(cudaMemcpyAsync(E.bins.p, bins.data(), bins.size() * sizeof(EllBin), cudaMemcpyHostToDevice, s));
    FSI_TRY(E.perm.alloc((size_t)n * 4));
    FSI_CUDA(cudaMemcpyAsync(E.perm.p, srows.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    DevBuf dbase, dstride;
    FSI_TRY(dbase.alloc((size_t)n * 8));
    FSI_TRY(dstride.alloc((size_t)n * 4));
    FSI_CUDA(cudaMemcpyAsync(dbase.p, base.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(dstride.p, rstride.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    FSI_TRY(E.col.alloc((size_t)E.size * 4));
    FSI_CUDA(cudaMemsetAsync(E.col.p, 0, (size_t)E.size * 4, s));
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    int32_t *ecol = E.col.as<int32_t>();
    if (A.val64.p) {
        FSI_TRY(E.val64.alloc((size_t)E.size * 8));
        FSI_CUDA(cudaMemsetAsync(E.val64.p, 0, (size_t)E.size * 8, s));
        ell_fill_subset_kernel<double><<<(unsigned)g, 256, 0, s>>>(n, E.perm.as<int32_t>(), A.ptr.as<int32_t>(),
                                                                   A.col.as<int32_t>(), A.val64.as<double>(), d_keep,
                                                                   dbase.as<int64_t>(), dstride.as<int32_t>(), ecol,
                                                                   E.val64.as<double>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
        ecol = nullptr;
    }
    if (A.val32.p) {
        FSI_TRY(E.val32.alloc((size_t)E.size * 4));
        FSI_CUDA(cudaMemsetAsync(E.val32.p, 0, (size_t)E.size * 4, s));
        ell_fill_subset_kernel<float><<<(unsigned)g, 256, 0, s>>>(n, E.perm.as<int32_t>(), A.ptr.as<int32_t>(),
                                                                  A.col.as<int32_t>(), A.val32.as<float>(), d_keep,
                                                                  dbase.as<int64_t>(), dstride.as<int32_t>(), ecol,
                                                                  E.val32.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    E.fbase = std::move(dbase);           // kept: refills after the CSR values change
    E.fstride = std::move(dstride);
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

// new CSR values, same pattern: re-fill the values of a row-subset copy in place
fsi_status ell_subset_refill(const DevCSR &A, DevEll &E, const uint8_t *d_keep, cudaStream_t s) {
    const int64_t n = E.perm.p ? (int64_t)(E.perm.bytes / 4) : 0;
    if (E.nbins == 0 || n == 0) return FSI_OK;
    if (!E.fbase.p) { set_error("ELL subset copy without a fill map"); return FSI_ERR_STATE; }
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (E.val64.p && A.val64.p) {
        ell_fill_subset_kernel<double><<<(unsigned)g, 256, 0, s>>>(n, E.perm.as<int32_t>(), A.ptr.as<int32_t>(),
                                                                   A.col.as<int32_t>(), A.val64.as<double>(), d_keep,
                                                                   E.fbase.as<int64_t>(), E.fstride.as<int32_t>(),
                                                                   nullptr, E.val64.as<double>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    if (E.val32.p && A.val32.p) {
        ell_fill_subset_kernel<float><<<(unsigned)g, 256, 0, s>>>(n, E.perm.as<int32_t>(), A.ptr.as<int32_t>(),
                                                                  A.col.as<int32_t>(), A.val32.as<float>(), d_keep,
                                                                  E.fbase.as<int64_t>(), E.fstride.as<int32_t>(),
                                                                  nullptr, E.val32.as<float>());
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    return FSI_OK;
}

// y[i] = b[i] - (E x)[i] on the rows of the subset copy E
template <class T>
fsi_status launch_ell_resid(const DevEll &E, const T *x, const T *b, T *y, cudaStream_t s) {
    if (E.nslabs == 0) return FSI_OK;
    const T *val = std::is_same<T, float>::value ? static_cast<const T *>(E.val32.p) : static_cast<const T *>(E.val64.p);
    if (!val) { set_error("ELL subset has no values in this precision"); return FSI_ERR_STATE; }
    return run_ell<T, T, T>(E, val, x, b, y, SPMV_RESID, s, (T *)nullptr);
}
template fsi_status launch_ell_resid<float>(const DevEll &, const float *, const float *, float *, cudaStream_t);
template fsi_status launch_ell_resid<double>(const DevEll &, const double *, const double *, double *, cudaStream_t);

template <class T>
fsi_status launch_axpy_clear(T *x, T *y, T a, int64_t n, cudaStream_t s) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) return FSI_OK;
    FSI_CUDA(launch_pdl(axpy_clear_kernel<T>, dim3((unsigned)g), dim3(256), 0, s, x, y, a, n));
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
template fsi_status launch_axpy_clear<float>(float *, float *, float, int64_t, cudaStream_t);
template fsi_status launch_axpy_clear<double>(double *, double *, double, int64_t, cudaStream_t);

}  // namespace fsi
