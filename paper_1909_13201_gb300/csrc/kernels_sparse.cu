// CSR sparse matrix-vector products: level residuals r = b - A x, the outer
// float64 product w = A z, restriction b_c = R r and prolongation x += P e.
//
// G threads cooperate on one row (G = 4..32 picked from the mean row length
// at set-up) so that the value and column streams are read in contiguous,
// coalesced runs; the partial sums are combined with warp shuffles.  Values
// and columns are streamed once (read-only, no L1 allocation); the gathered
// vector x stays in L2.  Accumulation is in the wider of the matrix and
// vector precisions.
#include <type_traits>

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
                                                   const TY *__restrict__ b, TY *__restrict__ y, int mode) {
    using AT = typename Acc<TA, TX>::type;
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
        }
        row += rows_per_grid;
    }
}

template <int G, int U, class TA, class TX, class TY>
fsi_status run(const DevCSR &A, const TA *val, const TX *x, const TY *b, TY *y, int mode, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (A.n_rows * G + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    spmv_kernel<G, U, TA, TX, TY><<<(unsigned)blocks, threads, 0, s>>>(A.n_rows, A.ptr.as<int32_t>(),
                                                                       A.col.as<int32_t>(), val, x, b, y, mode);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

}  // namespace

template <class TA, class TX, class TY>
fsi_status launch_spmv(const DevCSR &A, const TA *val, const TX *x, const TY *b, TY *y, int mode,
                       cudaStream_t s) {
    if (A.n_rows == 0) return FSI_OK;
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
        case 2: return run<GG, 2>(A, val, x, b, y, mode, s);        \
        case 4: return run<GG, 4>(A, val, x, b, y, mode, s);        \
        case 6: return run<GG, 6>(A, val, x, b, y, mode, s);        \
        default: return run<GG, 8>(A, val, x, b, y, mode, s);       \
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
                                                        const double *, double *, int, cudaStream_t);
template fsi_status launch_spmv<float, float, float>(const DevCSR &, const float *, const float *,
                                                     const float *, float *, int, cudaStream_t);

}  // namespace fsi
