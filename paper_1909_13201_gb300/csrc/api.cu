// C ABI of the solver (include/fsi.h): set-up of the hierarchy and the
// smoothers, the V-cycle (Sec. 3.2-3.3) and restarted flexible GMRES, the
// adjoint, and accessors.  Host code here only orders kernel launches and
// moves set-up data; every arithmetic step of a solve runs in the kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <type_traits>

#include <cublas_v2.h>

#include "context.h"

namespace fsi {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
// programmatic launches only inside a V-cycle, where every launch follows
// another kernel of the cycle (or the zeroing kernel at its top)
static thread_local int g_pdl_depth = 0;
struct PdlScope {
    PdlScope() { ++g_pdl_depth; }
    ~PdlScope() { --g_pdl_depth; }
};
bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("FSI_PDL");
        return !(e && e[0] == '0');
    }();
    return on && g_pdl_depth > 0;
}

namespace {

constexpr int NRED = 304;           // CTAs of the Krylov reductions (2 per SM)
constexpr int NDOT = 608;           // CTAs of the streaming first Gram-Schmidt pass (4 per SM)

// lanes per row of the SpMV kernel from the mean row length
int pick_group(int64_t rows, int64_t nnz) {
    const double avg = rows ? (double)nnz / (double)rows : 0.0;
    if (avg <= 3) return 1;
    if (avg <= 8) return 2;
    if (avg <= 20) return 4;
    if (avg <= 64) return 8;
    return 16;
}

fsi_status upload(DevBuf &d, const void *h, size_t bytes, cudaStream_t s) {
    FSI_TRY(d.alloc(bytes));
    if (bytes) FSI_CUDA(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
    return FSI_OK;
}

// host CSR (int64 ptr) -> device CSR (int32 ptr/col, float64 values)
fsi_status upload_csr(DevCSR &D, const HostCSR &H, cudaStream_t s) {
    if (H.nnz() > INT32_MAX) {
        set_error("operator has more than 2^31 nonzeros");
        return FSI_ERR_ARG;
    }
    D.n_rows = H.n_rows;
    D.n_cols = H.n_cols;
    D.nnz = H.nnz();
    std::vector<int32_t> p32(H.ptr.begin(), H.ptr.end());
    FSI_TRY(upload(D.ptr, p32.data(), p32.size() * 4, s));
    FSI_TRY(upload(D.col, H.col.data(), H.col.size() * 4, s));
    if (!H.val.empty()) FSI_TRY(upload(D.val64, H.val.data(), H.val.size() * 8, s));
    D.group = pick_group(D.n_rows, D.nnz);
    FSI_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    return FSI_OK;
}

fsi_status make_f32(DevCSR &D, cudaStream_t s) {
    if (D.val32.p || D.nnz == 0) return FSI_OK;
    FSI_TRY(D.val32.alloc((size_t)D.nnz * 4));
    FSI_TRY(launch_cast_f64_f32(D.val64.as<double>(), D.val32.as<float>(), D.nnz, s));
    return ell_fill_f32(D, s);
}

// device CSR -> host CSR (with values)
fsi_status download_csr(const DevCSR &D, HostCSR &H, cudaStream_t s) {
    std::vector<int32_t> p32(D.n_rows + 1);
    H.n_rows = D.n_rows;
    H.n_cols = D.n_cols;
    H.col.resize(D.nnz);
    H.val.resize(D.nnz);
    FSI_CUDA(cudaMemcpyAsync(p32.data(), D.ptr.p, p32.size() * 4, cudaMemcpyDeviceToHost, s));
    if (D.nnz) {
        FSI_CUDA(cudaMemcpyAsync(H.col.data(), D.col.p, (size_t)D.nnz * 4, cudaMemcpyDeviceToHost, s));
        FSI_CUDA(cudaMemcpyAsync(H.val.data(), D.val64.p, (size_t)D.nnz * 8, cudaMemcpyDeviceToHost, s));
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    H.ptr.assign(p32.begin(), p32.end());
    return FSI_OK;
}

void transpose_csr(const HostCSR &A, HostCSR &T) {
    T.n_rows = A.n_cols;
    T.n_cols = A.n_rows;
    T.ptr.assign(T.n_rows + 1, 0);
    for (int64_t k = 0; k < A.nnz(); ++k) T.ptr[A.col[k] + 1]++;
    for (int64_t r = 0; r < T.n_rows; ++r) T.ptr[r + 1] += T.ptr[r];
    T.col.resize(A.nnz());
    T.val.resize(A.nnz());
    std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t r = 0; r < A.n_rows; ++r)
        for (int64_t k = A.ptr[r]; k < A.ptr[r + 1]; ++k) {
            const int64_t q = pos[A.col[k]]++;
            T.col[q] = (int32_t)r;
            T.val[q] = A.val[k];
        }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

fsi_status read_flag(Context &cx, int *out) {
    FSI_CUDA(cudaMemcpyAsync(out, cx.flags.p, 4, cudaMemcpyDeviceToHost, cx.stream));
    FSI_CUDA(cudaStreamSynchronize(cx.stream));
    return FSI_OK;
}

// --------------------------------------------------------------- V-cycle
template <class T> const T *mval(const DevCSR &A);
template <> const float *mval<float>(const DevCSR &A) { return A.val32.as<float>(); }
template <> const double *mval<double>(const DevCSR &A) { return A.val64.as<double>(); }

// x += omega P2^{-1} r: Schwarz blocks and the Jacobi rows in one launch
// CUDA events around fine-level launches while profiling (fsi_profile)
cudaEvent_t take_event(Context &cx) {
    if (cx.ev_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = cx.ev_pool.back();
    cx.ev_pool.pop_back();
    return e;
}
struct ProfMark {
    Context &cx;
    int kind;
    bool on;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfMark(Context &c, int k, bool enable) : cx(c), kind(k), on(enable && c.profile) {
        if (on) {
            a = take_event(cx);
            b = take_event(cx);
            cudaEventRecord(a, cx.stream);
        }
    }
    ~ProfMark() {
        if (on) {
            cudaEventRecord(b, cx.stream);
            cx.ev_marks.push_back({kind, {a, b}});
        }
    }
};
// after the stream is idle: add the recorded durations to the totals
void collect_marks(Context &cx) {
    for (auto &m : cx.ev_marks) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, m.second.first, m.second.second);
        cx.prof_ms[m.first] += ms;
        cx.prof_n[m.first] += 1;
        cx.ev_pool.push_back(m.second.first);
        cx.ev_pool.push_back(m.second.second);
    }
    cx.ev_marks.clear();
}

// Locally multiplicative smoothing step (Sec. 3.2, multiplicative update
// formula, applied to each field system of P2): y = M r by the passes of the
// level in order (transposed: in reverse, with A_jj^{-T} and A_FF^T), where
// a pass corrects y on its blocks from r - A_FF y on its rows (the first pass
// of a field starts from y = 0 and reads r itself); then x += omega y and y is
// cleared for the next sweep.  P2 is block diagonal in the two field systems
// and each sweep reads and writes only its own system's rows of y and rr, so
// the velocity system's passes run on an auxiliary stream beside the
// displacement system's (forked from and joined back to the caller's stream).
template <class T>
fsi_status mult_smooth(Context &cx, LevelDev &L, const T *r, T *x, bool tr) {
    cudaStream_t s = cx.stream;
    if (tr && !L.mult_t_ready) {
        set_error("transposed multiplicative sweep needs the transposed operators (fsi_adjoint builds them)");
        return FSI_ERR_STATE;
    }
    T *y = L.y.as<T>(), *rr = L.rr.as<T>();
    const int np = (int)L.passes.size();
    const bool two = L.fj.aux != nullptr;
    if (two) {
        FSI_CUDA(cudaEventRecord(L.fj.fork, s));
        FSI_CUDA(cudaStreamWaitEvent(L.fj.aux, L.fj.fork, 0));
    }
    bool started[2] = {false, false};
    for (int q = 0; q < np; ++q) {
        const SweepPass &P = L.passes[tr ? np - 1 - q : q];
        cudaStream_t sp = (two && P.field == 1) ? L.fj.aux : s;
        const T *src = r;
        if (started[P.field]) {
            FSI_TRY(launch_ell_resid<T>(tr ? P.ell_t : P.ell, y, r, rr, sp));
            src = rr;
        }
        started[P.field] = true;
        FSI_TRY(launch_block_apply<T>(L, src, y, (T)1, tr ? 1 : 0, sp, P.it0, P.it1));
    }
    if (two) {
        FSI_CUDA(cudaEventRecord(L.fj.join, L.fj.aux));
        FSI_CUDA(cudaStreamWaitEvent(s, L.fj.join, 0));
    }
    return launch_axpy_clear<T>(x, y, (T)cx.omega, L.n, s);
}

template <class T>
fsi_status smooth_apply(Context &cx, LevelDev &L, const T *r, T *x, bool tr, bool fine = false) {
    ProfMark pm(cx, 0, fine);
    if (L.mult) return mult_smooth<T>(cx, L, r, x, tr);
    return launch_block_apply<T>(L, r, x, (T)cx.omega, tr ? 1 : 0, cx.stream);
}

// x_l = M_l^{-1} b_l from a zero guess (transposed cycle if tr)
template <class T>
fsi_status vcycle(Context &cx, Problem &pb, int l, const T *b, T *x, bool tr, bool x_zeroed = false) {
    cudaStream_t s = cx.stream;
    const bool cz = cx.cascade != 0;        // swapped cascade: the two system blocks only
    if (l == 0) {
        // transposed cycle: the stored transpose, read row by row like the forward
        // product (a column-by-column product of the row-major inverse takes 20x longer)
        const DevBuf &inv = cz ? pb.coarse_inv_c : pb.coarse_inv;
        const DevBuf &inv_t = cz ? pb.coarse_inv_ct : pb.coarse_inv_t;
        if (tr && inv_t.p) return launch_dense_gemv<T>(inv_t.as<double>(), pb.n0, b, x, 0, s);
        return launch_dense_gemv<T>(inv.as<double>(), pb.n0, b, x, tr ? 1 : 0, s);
    }
    LevelDev &L = pb.dev[l];
    LevelDev &C = pb.dev[l - 1];
    const DevCSR &A = tr ? (cz ? L.ATc : L.AT) : (cz ? L.Ac : L.A);
    const DevCSR &Rm = tr ? L.PT : (cz ? L.Rc : L.R);     // restriction
    const DevCSR &Pm = tr ? (cz ? L.RTc : L.RT) : L.P;    // prolongation
    const int npre = tr ? cx.nu_post : cx.nu_pre, npost = tr ? cx.nu_pre : cx.nu_post;
    const bool fine = l == (int)pb.dev.size() - 1;
    T *r = L.r.as<T>();
    if (!x_zeroed) FSI_TRY(launch_zero<T>(x, L.n, s));
    PdlScope pdl;
    for (int k = 0; k < npre; ++k) {
        if (k == 0) {
            FSI_TRY(smooth_apply<T>(cx, L, b, x, tr, fine));
        } else {
            FSI_TRY(launch_spmv<T, T, T>(A, mval<T>(A), x, b, r, SPMV_RESID, s));
            FSI_TRY(smooth_apply<T>(cx, L, r, x, tr, fine));
        }
    }
    {
        ProfMark pm(cx, 1, fine);
        FSI_TRY(launch_spmv<T, T, T>(A, mval<T>(A), x, b, r, SPMV_RESID, s));
    }
    {
        ProfMark pm(cx, 4, fine);
        // b_{l-1} = R r, and x_{l-1} = 0 in the same launch (level 0 is written whole)
        FSI_TRY(launch_spmv<T, T, T>(Rm, mval<T>(Rm), r, (const T *)nullptr, C.b.as<T>(), SPMV_SET, s,
                                     l - 1 > 0 ? C.x.as<T>() : (T *)nullptr));
    }
    FSI_TRY(vcycle<T>(cx, pb, l - 1, C.b.as<T>(), C.x.as<T>(), tr, true));
    {
        ProfMark pm(cx, 5, fine);
        FSI_TRY(launch_spmv<T, T, T>(Pm, mval<T>(Pm), C.x.as<T>(), (const T *)nullptr, x, SPMV_ADD, s));
    }
    for (int k = 0; k < npost; ++k) {
        {
            ProfMark pm(cx, 1, fine);
            FSI_TRY(launch_spmv<T, T, T>(A, mval<T>(A), x, b, r, SPMV_RESID, s));
        }
        FSI_TRY(smooth_apply<T>(cx, L, r, x, tr, fine));
    }
    return FSI_OK;
}

// ------------------------------------------------------------ workspace
// duration of the last batch-graph launch (every system of the batch reports it)
float batch_ms_last = 0.f;

// bumped whenever a problem's graphs are dropped (workspace or smoothers
// changed): a batch graph captured under an older epoch is stale
std::atomic<int64_t> g_graph_epoch{0};

void drop_graphs(Problem &pb) {
    ++g_graph_epoch;
    for (auto &v : pb.graphs) {
        for (auto &ge : v)
            if (ge) cudaGraphExecDestroy(ge);
        v.clear();
    }
    for (auto &v : pb.graph_kernels) v.clear();
    for (int d = 0; d < 2; ++d) {
        if (pb.solve_graph[d]) cudaGraphExecDestroy(pb.solve_graph[d]);
        pb.solve_graph[d] = nullptr;
        pb.solve_graph_m[d] = 0;
    }
}

fsi_status ensure_workspace(Context &cx, Problem &pb, int m) {
    if (pb.m_alloc >= m) return FSI_OK;
    drop_graphs(pb);
    const int64_t n = pb.dev.back().n;
    FSI_TRY(pb.V.alloc((size_t)n * (m + 1) * 8));
    FSI_TRY(pb.V32.alloc((size_t)n * (m + 1) * 4));
    FSI_TRY(pb.Z.alloc((size_t)n * m * 8));     // float64: the outer SpMV reads it without conversions
    FSI_TRY(pb.H.alloc((size_t)(m + 1) * m * 8));
    FSI_TRY(pb.g.alloc((size_t)(m + 2) * 8));
    FSI_TRY(pb.cs.alloc((size_t)(m + 1) * 8));
    FSI_TRY(pb.sn.alloc((size_t)(m + 1) * 8));
    FSI_TRY(pb.y.alloc((size_t)(m + 1) * 8));
    FSI_TRY(pb.w.alloc((size_t)n * 8));
    FSI_TRY(pb.rvec.alloc((size_t)n * 8));
    FSI_TRY(pb.partials.alloc((size_t)NDOT * 65 * 8));
    FSI_TRY(pb.scal.alloc(64 * 8));
    FSI_TRY(pb.h1.alloc((size_t)(m + 1) * 8));
    FSI_TRY(pb.h2.alloc((size_t)(m + 1) * 8));
    pb.m_alloc = m;
    return FSI_OK;
}

// ||v||^2 into scal[slot] (device)
fsi_status norm2(Context &cx, Problem &pb, const double *v, int64_t n, int slot) {
    FSI_TRY(launch_mdot(v, n, 1, v, n, pb.partials.as<double>(), NRED, cx.stream));
    return launch_reduce_partials(pb.partials.as<double>(), NRED, 1, pb.scal.as<double>() + slot, 0, cx.stream);
}


// --------------------------------------------------------------- FGMRES
// Right-preconditioned FGMRES(m) with CGS2 Arnoldi and Givens rotations;
// converged when the float64 true residual ||b - A x|| <= rtol ||b||.
//
// The method is written as a resumable state machine so that several
// independent problems advance together: each round enqueues one step of
// every active run on the run's own stream (asynchronously, ending with a
// device-to-host copy of the step's scalars into the run's pinned slot),
// waits for all streams, and then lets every run read its scalars and pick
// its next step.  One problem is the plain sequential solve.
struct Run {
    Problem *pb = nullptr;
    const double *b = nullptr;
    double *x = nullptr;
    bool tr = false;
    fsi_solve_opts o{};
    enum { NORM_B, START, CYCLE, STEP, DONE } phase = NORM_B;
    int its = 0, j = 0, k = 0;
    double bnorm = 0, beta = 0;
    fsi_status status = FSI_OK;
    fsi_solve_stats st{};
    std::chrono::steady_clock::time_point t0;
};

// one Arnoldi step j of problem pb on stream s: z_j = M^{-1} v_j, w = A z_j,
// CGS2, Givens, the scalars (estimate, h_{j+1,j}, ||A z_j||, flags) to the
// pinned slot, and v_{j+1} = w / h_{j+1,j}.  Fixed buffers only, so it is
// captured once per j as a CUDA graph and replayed in later solves.
template <class T>
fsi_status issue_step(Context &cx, Problem &pb, int j, int m, bool tr) {
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    const int L = (int)pb.dev.size();
    const DevCSR &A = tr ? F.AT : F.A;
    double *V = pb.V.as<double>(), *H = pb.H.as<double>(), *g = pb.g.as<double>();
    double *w = pb.w.as<double>(), *scal = pb.scal.as<double>(), *Z = pb.Z.as<double>();
    double *vj = V + (size_t)j * n;
    double *zj = Z + (size_t)j * n;
    if (std::is_same<T, double>::value) {
        FSI_TRY(vcycle<T>(cx, pb, L - 1, reinterpret_cast<const T *>(vj), reinterpret_cast<T *>(zj), tr));
    } else {
        T *bfine = F.b.as<T>();
        FSI_TRY(launch_cast_f64_f32(vj, reinterpret_cast<float *>(bfine), n, s));
        FSI_TRY(vcycle<T>(cx, pb, L - 1, bfine, F.x.as<T>(), tr));
        FSI_TRY(launch_cast_f32_f64(reinterpret_cast<const float *>(F.x.as<T>()), zj, n, s));
    }
    // float64 A z_j: the row-scaled systems reach 1e-8 only a little above
    // their attainable accuracy, so this product keeps full float64 rounding
    {
        ProfMark pm(cx, 2, true);
        FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), zj, (const double *)nullptr, w,
                                                    SPMV_SET, s));
    }
    const int nv = j + 1;
    double *part = pb.partials.as<double>(), *h1 = pb.h1.as<double>(), *h2 = pb.h2.as<double>();
    float *V32 = cx.precision != FSI_FP64 ? pb.V32.as<float>() : nullptr;
    {
        ProfMark pm(cx, 7, true);       // first pass: bytes of the basis (copy) and w
        if (cx.profile) cx.prof_work[7] += (double)nv * n * (V32 ? 4.0 : 8.0) + (double)n * 8.0;
        if (V32) FSI_TRY(launch_mdot32(V32, n, nv, w, n, part, NDOT, s));
        else FSI_TRY(launch_mdot(V, n, nv, w, n, part, NDOT, s));
    }
    {
        PdlScope pdl;                   // programmatic launches up to the Givens step
        FSI_TRY(launch_reduce_partials(part, NDOT, nv, h1, 0, s));
        {
            ProfMark pm(cx, 6, true);       // float64 update (+ float64 dots): nv (2 nv) FMAs per row
            if (cx.profile) {
                cx.prof_work[6] += (V32 ? 1.0 : 2.0) * nv * n;
                cx.prof_gs64_bytes += (double)nv * n * (V32 ? 12.0 : 8.0) + 16.0 * n;   // V (+ V32), w in and out
            }
            FSI_TRY(launch_update_dot(w, V, n, nv, h1, n, part, NRED, 0, s, nullptr, V32));
        }
        FSI_TRY(launch_reduce_partials(part, NRED, nv, h2, 0, s));
        {
            ProfMark pm(cx, 6, true);       // float64 update + norm: nv + 1 FMAs per row
            if (cx.profile) {
                cx.prof_work[6] += (nv + 1.0) * n;
                cx.prof_gs64_bytes += (double)nv * n * 8.0 + 16.0 * n;
            }
            FSI_TRY(launch_update_dot(w, V, n, nv, h2, n, part, NRED, 1, s));
        }
        FSI_TRY(launch_reduce_partials(part, NRED, 1, scal + 7, 0, s));
        FSI_TRY(launch_givens(H, m + 1, j, h1, h2, scal + 7, pb.cs.as<double>(), pb.sn.as<double>(), g, scal, s));
    }
    FSI_CUDA(cudaMemcpyAsync(pb.h_scal, scal, 5 * 8, cudaMemcpyDeviceToHost, s));
    FSI_TRY(launch_scale_copy(w, V + (size_t)(j + 1) * n, scal, 1, n, s, nullptr, 0,
                              V32 ? V32 + (size_t)(j + 1) * n : nullptr));
    return FSI_OK;
}

// enqueue ||v||^2 -> scal[slot] and its copy to the pinned slot
fsi_status norm2_to_host(Context &cx, Problem &pb, const double *v, int64_t n, int slot) {
    FSI_TRY(norm2(cx, pb, v, n, slot));
    FSI_CUDA(cudaMemcpyAsync(pb.h_scal + slot, pb.scal.as<double>() + slot, 8, cudaMemcpyDeviceToHost, cx.stream));
    return FSI_OK;
}

template <class T>
fsi_status enqueue(Context &cx, Run &R) {
    Problem &pb = *R.pb;
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    const int m = R.o.restart;
    const DevCSR &A = R.tr ? F.AT : F.A;
    double *r = pb.rvec.as<double>();
    switch (R.phase) {
        case Run::NORM_B:
            return norm2_to_host(cx, pb, R.b, n, 5);
        case Run::START:
            if (!R.o.use_x0) FSI_CUDA(cudaMemsetAsync(R.x, 0, (size_t)n * 8, s));
            FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), R.x, R.b, r, SPMV_RESID, s));
            return norm2_to_host(cx, pb, r, n, 6);
        case Run::CYCLE:
            FSI_TRY(launch_init_basis(r, pb.V.as<double>(), pb.g.as<double>(), m, pb.scal.as<double>() + 6, n, s,
                                      nullptr, 0, cx.precision != FSI_FP64 ? pb.V32.as<float>() : nullptr));
            R.j = 0;
            // fall through: the first step of the cycle goes in the same round
        case Run::STEP: {
            const int j = R.j;
            const bool graphs = cx.use_graphs && !cx.profile && s != nullptr;
            auto &gexec = pb.graphs[R.tr ? 1 : 0];
            auto &gkern = pb.graph_kernels[R.tr ? 1 : 0];
            if (!graphs) return issue_step<T>(cx, pb, j, m, R.tr);
            if ((int)gexec.size() != m) {
                for (auto &ge : gexec)
                    if (ge) cudaGraphExecDestroy(ge);
                gexec.assign(m, nullptr);
                gkern.assign(m, 0);
            }
            if (!gexec[j]) {
                const int64_t before = launches_so_far();
                cudaGraph_t gr = nullptr;
                FSI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                fsi_status cs = issue_step<T>(cx, pb, j, m, R.tr);
                cudaError_t ce = cudaStreamEndCapture(s, &gr);
                if (cs != FSI_OK) {
                    if (gr) cudaGraphDestroy(gr);
                    return cs;
                }
                FSI_CUDA(ce);
                FSI_CUDA(cudaGraphInstantiate(&gexec[j], gr, 0));
                cudaGraphDestroy(gr);
                gkern[j] = launches_so_far() - before;
                count_launch(-(int)gkern[j]);        // captured, not run
            }
            FSI_CUDA(cudaGraphLaunch(gexec[j], s));
            count_launch((int)gkern[j]);
            return FSI_OK;
        }
        default:
            return FSI_OK;
    }
}

// end of a cycle: x += Z y, true residual
fsi_status enqueue_end_cycle(Context &cx, Run &R) {
    Problem &pb = *R.pb;
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    const int m = R.o.restart;
    const DevCSR &A = R.tr ? F.AT : F.A;
    FSI_TRY(launch_backsolve(pb.H.as<double>(), m + 1, R.k, pb.g.as<double>(), pb.y.as<double>(), s));
    FSI_TRY(launch_combine<double>(R.x, pb.Z.as<double>(), n, R.k, pb.y.as<double>(), n, s));
    FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), R.x, R.b, pb.rvec.as<double>(), SPMV_RESID, s));
    return norm2_to_host(cx, pb, pb.rvec.as<double>(), n, 6);
}

void finish(Run &R, fsi_status status) {
    R.phase = Run::DONE;
    R.st.iterations = R.its;
    R.st.rN = R.beta;
    R.st.rel_residual = R.bnorm > 0 ? R.beta / R.bnorm : 0.0;
    R.st.converged = R.bnorm == 0.0 || R.beta <= R.o.rtol * R.bnorm;
    R.st.rho = (R.its > 0 && R.st.r0 > 0) ? std::pow(R.beta / R.st.r0, 1.0 / R.its) : 0.0;
    if (status == FSI_OK && !std::isfinite(R.beta)) {
        status = FSI_ERR_NONFINITE;
        set_error("non-finite residual");
    }
    if (status == FSI_OK && !R.st.converged) {
        status = FSI_ERR_NOT_CONVERGED;
        set_error("FGMRES did not reach rtol within max_iters");
    }
    R.status = status;
    R.st.status = status;
    R.st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - R.t0).count();
}

// after the round's streams are idle: read the scalars, choose the next step
fsi_status advance(Context &cx, Run &R, bool &end_cycle) {
    const double *hs = R.pb->h_scal;
    end_cycle = false;
    switch (R.phase) {
        case Run::NORM_B:
            R.bnorm = std::sqrt(hs[5]);
            if (!std::isfinite(R.bnorm)) {
                set_error("right-hand side has a non-finite norm");
                R.beta = NAN;
                finish(R, FSI_ERR_NONFINITE);
            } else if (R.bnorm == 0.0) {
                FSI_CUDA(cudaMemsetAsync(R.x, 0, (size_t)R.pb->dev.back().n * 8, cx.stream));
                R.beta = 0.0;
                finish(R, FSI_OK);
            } else {
                R.phase = Run::START;
            }
            return FSI_OK;
        case Run::START:
            R.beta = std::sqrt(hs[6]);
            R.st.r0 = R.beta;
            break;
        case Run::CYCLE:
        case Run::STEP: {
            ++R.its;
            R.k = R.j + 1;
            const double est = hs[0], hn = hs[1], wn = hs[2];
            if (hs[4] != 0.0) {
                set_error("non-finite value in the Arnoldi process");
                R.beta = NAN;
                finish(R, FSI_ERR_NONFINITE);
                return FSI_OK;
            }
            if (est <= R.o.rtol * R.bnorm || hn <= 1e-14 * wn || R.its >= R.o.max_iters || R.k == R.o.restart) {
                end_cycle = true;               // caller enqueues x update + true residual
            } else {
                R.j = R.j + 1;
                R.phase = Run::STEP;
            }
            return FSI_OK;
        }
        default:
            return FSI_OK;
    }
    // after a true residual (start of solve or end of a cycle)
    if (R.beta > R.o.rtol * R.bnorm && R.its < R.o.max_iters && std::isfinite(R.beta)) R.phase = Run::CYCLE;
    else finish(R, FSI_OK);
    return FSI_OK;
}

template <class T>
fsi_status run_batch(Context &cx, std::vector<Run> &runs) {
    cudaStream_t user = cx.stream;
    FSI_CUDA(cudaMemsetAsync(cx.flags.as<int>() + 2, 0, 4, user));   // kernel error word
    for (auto &R : runs) {
        FSI_TRY(ensure_workspace(cx, *R.pb, R.o.restart));
        R.t0 = std::chrono::steady_clock::now();
        R.st = fsi_solve_stats();
        // every problem stream starts after the work queued on the caller's stream
        FSI_CUDA(cudaEventRecord(cx.ev_in, user));
        FSI_CUDA(cudaStreamWaitEvent(R.pb->stream, cx.ev_in, 0));
    }
    fsi_status err = FSI_OK;
    std::vector<char> residual_next(runs.size(), 0);
    while (err == FSI_OK) {
        bool any = false;
        for (size_t i = 0; i < runs.size(); ++i) {
            Run &R = runs[i];
            if (R.phase == Run::DONE) continue;
            any = true;
            cx.stream = R.pb->stream;
            fsi_status e = residual_next[i] ? enqueue_end_cycle(cx, R) : enqueue<T>(cx, R);
            if (e != FSI_OK) { err = e; break; }
        }
        cx.stream = user;
        if (!any || err != FSI_OK) break;
        for (auto &R : runs)
            if (R.phase != Run::DONE) {
                cudaError_t ce = cudaStreamSynchronize(R.pb->stream);
                if (ce != cudaSuccess) {
                    set_error(std::string("solve stream: ") + cudaGetErrorString(ce));
                    err = FSI_ERR_CUDA;
                }
            }
        if (err != FSI_OK) break;
        for (size_t i = 0; i < runs.size(); ++i) {
            Run &R = runs[i];
            if (R.phase == Run::DONE) continue;
            cx.stream = R.pb->stream;
            if (residual_next[i]) {
                // a cycle ended: hs[6] holds the new true residual
                residual_next[i] = 0;
                R.st.cycles++;
                R.beta = std::sqrt(R.pb->h_scal[6]);
                if (R.beta > R.o.rtol * R.bnorm && R.its < R.o.max_iters && std::isfinite(R.beta))
                    R.phase = Run::CYCLE;
                else
                    finish(R, FSI_OK);
                continue;
            }
            bool end_cycle = false;
            fsi_status e = advance(cx, R, end_cycle);
            if (e != FSI_OK) { err = e; break; }
            if (end_cycle) residual_next[i] = 1;
        }
        cx.stream = user;
    }
    cx.stream = user;
    for (auto &R : runs) {
        FSI_CUDA(cudaEventRecord(cx.ev_out, R.pb->stream));
        FSI_CUDA(cudaStreamWaitEvent(user, cx.ev_out, 0));
        if (R.phase != Run::DONE) finish(R, err == FSI_OK ? FSI_ERR_STATE : err);
    }
    if (!cx.ev_marks.empty()) {
        for (auto &R : runs) cudaStreamSynchronize(R.pb->stream);
        collect_marks(cx);
    }
    return err;
}

fsi_status check_opts(const fsi_solve_opts *o) {
    if (!o) { set_error("opts is NULL"); return FSI_ERR_ARG; }
    if (!(o->rtol > 0.0) || o->restart < 1 || o->restart > 64 || o->max_iters < 1) {
        set_error("solve options out of range (rtol > 0, 1 <= restart <= 64, max_iters >= 1)");
        return FSI_ERR_ARG;
    }
    return FSI_OK;
}

fsi_status build_transposes(Context &cx, Problem &pb) {
    if (pb.transposes_ready) return FSI_OK;
    cudaStream_t s = cx.stream;
    drop_graphs(pb);     // transposed copies are (re)allocated below
    if (!pb.coarse_inv_t.p) {
        FSI_TRY(pb.coarse_inv_t.alloc((size_t)pb.n0 * pb.n0 * 8));
        FSI_TRY(launch_transpose(pb.coarse_inv.as<double>(), pb.n0, pb.coarse_inv_t.as<double>(), s));
    }
    if (cx.cascade) {
        FSI_TRY(pb.coarse_inv_ct.alloc((size_t)pb.n0 * pb.n0 * 8));
        FSI_TRY(launch_transpose(pb.coarse_inv_c.as<double>(), pb.n0, pb.coarse_inv_ct.as<double>(), s));
    }
    for (size_t l = 0; l < pb.dev.size(); ++l) {
        LevelDev &L = pb.dev[l];
        HostCSR A, AT;
        FSI_TRY(download_csr(L.A, A, s));
        transpose_csr(A, AT);
        FSI_TRY(upload_csr(L.AT, AT, s));
        FSI_TRY(build_ell(L.AT, s, cx.probs.size() > 1, cx.ell_lanes));
        if (cx.cascade) {
            HostCSR Ac, ATc;
            FSI_TRY(download_csr(L.Ac, Ac, s));
            transpose_csr(Ac, ATc);
            FSI_TRY(upload_csr(L.ATc, ATc, s));
            FSI_TRY(build_ell(L.ATc, s, cx.probs.size() > 1, cx.ell_lanes));
            L.ATc.val32.release();
            if (cx.precision != FSI_FP64) FSI_TRY(make_f32(L.ATc, s));
            if (l >= 1) {
                HostCSR Rc, RTc;
                FSI_TRY(download_csr(L.Rc, Rc, s));
                transpose_csr(Rc, RTc);
                FSI_TRY(upload_csr(L.RTc, RTc, s));
                FSI_TRY(build_ell(L.RTc, s, cx.probs.size() > 1, cx.ell_lanes));
                L.RTc.val32.release();
                if (cx.precision != FSI_FP64) FSI_TRY(make_f32(L.RTc, s));
            }
        }
        if (l >= 1) {
            HostCSR PT, RT;
            transpose_csr(pb.hP[l], PT);
            transpose_csr(pb.hR[l], RT);
            FSI_TRY(upload_csr(L.PT, PT, s));
            FSI_TRY(upload_csr(L.RT, RT, s));
            FSI_TRY(build_ell(L.PT, s, cx.probs.size() > 1, cx.ell_lanes));
            FSI_TRY(build_ell(L.RT, s, cx.probs.size() > 1, cx.ell_lanes));
        }
        if (cx.precision != FSI_FP64) {
            FSI_TRY(make_f32(L.AT, s));
            if (l >= 1) {
                FSI_TRY(make_f32(L.PT, s));
                FSI_TRY(make_f32(L.RT, s));
            }
        }
        if (L.mult) {
            // A_FF^T on every pass's rows (the field masks are symmetric)
            for (auto &P : L.passes)
                FSI_TRY(build_ell_subset(L.AT, AT, P.rows, L.h_keep[P.field], L.keep[P.field].as<uint8_t>(), P.ell_t,
                                         s, cx.probs.size() > 1));
            L.mult_t_ready = true;
        }
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    pb.transposes_ready = true;
    return FSI_OK;
}

fsi_status setup_problem(Context &cx, Problem &pb, const fsi_problem &in) {
    cudaStream_t s = cx.stream;
    ProblemDesc &d = pb.desc;
    d.dim = in.dim;
    d.n_fine = in.n_fine;
    d.n_levels = in.n_levels;
    d.bc_preset = in.bc_preset;
    d.mu_s = in.mu_s; d.lambda_s = in.lambda_s; d.rho_s = in.rho_s;
    d.rho_f = in.rho_f; d.mu_f = in.mu_f; d.dt = in.dt;
    d.nonlinear = cx.nonlinear;
    if (!in.material || !in.advection) { set_error("material/advection is NULL"); return FSI_ERR_ARG; }
    if (in.dim != 2 && in.dim != 3) { set_error("dim must be 2 or 3"); return FSI_ERR_ARG; }
    if (in.n_fine < 1 || in.n_fine > 4096) { set_error("n_fine out of range"); return FSI_ERR_ARG; }
    if (!(in.dt > 0) || !(in.lambda_s > 0) || !(in.mu_s > 0) || !(in.mu_f > 0)) {
        set_error("coefficients must be positive");
        return FSI_ERR_ARG;
    }
    int64_t nel = 1, nq2 = 1;
    for (int k = 0; k < in.dim; ++k) { nel *= in.n_fine; nq2 *= 2 * (int64_t)in.n_fine + 1; }
    d.material.assign(in.material, in.material + nel);
    d.advection.assign(in.advection, in.advection + (size_t)in.dim * nq2);
    std::string err = build_levels(d, pb.host);
    if (!err.empty()) { set_error(err); return FSI_ERR_ARG; }
    const int L = d.n_levels;
    pb.dev.resize(L);
    pb.hP.resize(L);
    pb.hR.resize(L);
    if (cx.host_only) {
        for (int l = 1; l < L; ++l) {
            build_prolongation(pb.host[l], pb.host[l - 1], pb.hP[l]);
            build_restriction(pb.hP[l], pb.host[l], pb.host[l - 1], cx.restriction == 1, pb.hR[l]);
        }
        for (int l = 0; l < L; ++l) {
            pb.dev[l].n = pb.host[l].n_dofs;
            pb.dev[l].A.nnz = pb.host[l].pattern.nnz();
            if (l >= 1 && cx.patch >= 1) {
                LevelDev &D = pb.dev[l];
                std::vector<int32_t> tags;
                build_blocks(pb.host[l], cx.patch, D.h_blk_ptr, D.h_blk_idx, false, &tags);
                sweep_passes(pb.host[l], cx.patch, tags, D.h_pass);
                D.n_blocks = (int64_t)D.h_blk_ptr.size() - 1;
                D.max_block = 0;
                for (int64_t j = 0; j < D.n_blocks; ++j)
                    D.max_block = std::max(D.max_block, D.h_blk_ptr[j + 1] - D.h_blk_ptr[j]);
            }
        }
        return FSI_OK;
    }
    RefTables ref = make_ref_tables(d.dim);
    FSI_CUDA(cudaStreamCreateWithFlags(&pb.stream, cudaStreamNonBlocking));
    FSI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&pb.h_scal), 16 * 8));
    FSI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&pb.h_fg), 2 * sizeof(FgState)));
    pb.h_fg[0] = FgState();
    pb.h_fg[1] = FgState();
    FSI_TRY(pb.fg.alloc(sizeof(FgState)));
    FSI_CUDA(cudaEventCreate(&pb.ev_a));
    FSI_CUDA(cudaEventCreate(&pb.ev_b));
    for (int l = 0; l < L; ++l) {
        LevelHost &H = pb.host[l];
        LevelDev &D = pb.dev[l];
        D.n = H.n_dofs;
        FSI_TRY(upload_csr(D.A, H.pattern, s));
        FSI_TRY(D.A.val64.alloc((size_t)D.A.nnz * 8));
        FSI_TRY(launch_assemble(H, d, ref, D.A, false, D.A.val64.as<double>(), s));
        FSI_TRY(build_ell(D.A, s, cx.probs.size() > 1, cx.ell_lanes));
        FSI_TRY(upload(D.fixed, H.fixed.data(), H.fixed.size(), s));
        if (l >= 1) {
            build_prolongation(H, pb.host[l - 1], pb.hP[l]);
            build_restriction(pb.hP[l], H, pb.host[l - 1], cx.restriction == 1, pb.hR[l]);
            FSI_TRY(upload_csr(D.P, pb.hP[l], s));
            FSI_TRY(upload_csr(D.R, pb.hR[l], s));
            FSI_TRY(build_ell(D.P, s, cx.probs.size() > 1, cx.ell_lanes));
            FSI_TRY(build_ell(D.R, s, cx.probs.size() > 1, cx.ell_lanes));
        }
    }
    // dA/dmu_s on the fine pattern (adjoint gradient)
    {
        LevelDev &F = pb.dev.back();
        FSI_TRY(pb.dA_mu.alloc((size_t)F.A.nnz * 8));
        FSI_TRY(launch_assemble(pb.host.back(), d, ref, F.A, true, pb.dA_mu.as<double>(), s));
    }
    // coarse direct solve: float64 inverse of A_0 (Gauss-Jordan, partial pivoting)
    pb.n0 = pb.dev[0].n;
    FSI_TRY(pb.coarse_inv.alloc((size_t)pb.n0 * pb.n0 * 8));
    FSI_CUDA(cudaMemsetAsync(cx.flags.p, 0, 16, s));
    FSI_TRY(coarse_invert(pb.dev[0].A, pb.n0, pb.coarse_inv.as<double>(), cx.flags.as<int>(), s));
    int flag = 0;
    FSI_TRY(read_flag(cx, &flag));
    if (flag) {
        set_error("coarse-level operator is singular");
        return FSI_ERR_ZERO_PIVOT;
    }
    return FSI_OK;
}

// Swapped cascade (Sec. 5, future work): the cycle runs on the two system
// blocks of every operator -- the displacement system [d^s, d^f, p^s] (J2
// dofs before off[3]) and the velocity system [u^s, u^f, p^f] -- so one
// V-cycle is blockdiag(GMG_d, GMG_u).  Built once per problem: A_l and R_l
// without their cross-system entries, and the float64 inverse of the coarse
// block-diagonal operator.  P_l couples no systems (checked).
HostCSR split_systems(const HostCSR &M, int64_t row_off3, int64_t col_off3) {
    HostCSR out;
    out.n_rows = M.n_rows;
    out.n_cols = M.n_cols;
    out.ptr.assign(1, 0);
    for (int64_t i = 0; i < M.n_rows; ++i) {
        const bool ri = i >= row_off3;
        for (int64_t k = M.ptr[i]; k < M.ptr[i + 1]; ++k) {
            if (((int64_t)M.col[k] >= col_off3) != ri) continue;
            out.col.push_back(M.col[k]);
            out.val.push_back(M.val[k]);
        }
        out.ptr.push_back((int64_t)out.col.size());
    }
    return out;
}

fsi_status build_cascade(Context &cx, Problem &pb) {
    if (pb.cascade_ready) return FSI_OK;
    cudaStream_t s = cx.stream;
    const bool conc = cx.probs.size() > 1;
    for (size_t l = 0; l < pb.dev.size(); ++l) {
        LevelDev &L = pb.dev[l];
        const LevelHost &H = pb.host[l];
        HostCSR A;
        FSI_TRY(download_csr(L.A, A, s));
        FSI_TRY(upload_csr(L.Ac, split_systems(A, H.off[3], H.off[3]), s));
        FSI_TRY(build_ell(L.Ac, s, conc, cx.ell_lanes));
        L.Ac.val32.release();
        if (l >= 1) {
            const LevelHost &Hc = pb.host[l - 1];
            const HostCSR &P = pb.hP[l];
            for (int64_t i = 0; i < P.n_rows; ++i)
                for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k)
                    if ((i >= H.off[3]) != ((int64_t)P.col[k] >= Hc.off[3])) {
                        set_error("prolongation couples the displacement and velocity systems");
                        return FSI_ERR_STATE;
                    }
            FSI_TRY(upload_csr(L.Rc, split_systems(pb.hR[l], Hc.off[3], H.off[3]), s));
            FSI_TRY(build_ell(L.Rc, s, conc, cx.ell_lanes));
            L.Rc.val32.release();
        }
    }
    FSI_TRY(pb.coarse_inv_c.alloc((size_t)pb.n0 * pb.n0 * 8));
    FSI_CUDA(cudaMemsetAsync(cx.flags.p, 0, 16, s));
    FSI_TRY(coarse_invert(pb.dev[0].Ac, pb.n0, pb.coarse_inv_c.as<double>(), cx.flags.as<int>(), s));
    int flag = 0;
    FSI_TRY(read_flag(cx, &flag));
    if (flag) {
        set_error("coarse-level system blocks are singular");
        return FSI_ERR_ZERO_PIVOT;
    }
    pb.cascade_ready = true;
    return FSI_OK;
}

// the smoother options a set-up was built with
std::vector<double> smoother_signature(const Context &cx) {
    return {(double)cx.precision, (double)cx.patch, cx.omega, (double)cx.nu_pre, (double)cx.nu_post,
            (double)cx.factor, (double)cx.variant, (double)cx.mult_levels, (double)cx.cascade,
            (double)cx.ell_lanes};
}

// Gather and invert the Schwarz blocks of level l (l >= 1) with the
// context's factor method into the level's existing inverse storage.
// (launch only, on stream s; flags accumulate in cx.flags)
fsi_status launch_level_inversion(Context &cx, Problem &pb, size_t l, cudaStream_t s) {
    LevelDev &D = pb.dev[l];
    const LevelHost &H = pb.host[l];
    const int store = D.inv_store;
    int method = cx.factor;
    if (method == FSI_FACTOR_AUTO) method = store == 0 ? FSI_FACTOR_FP64 : FSI_FACTOR_TF32;
    {
        ProfMark pm(cx, 3, l + 1 == pb.dev.size());
        // monolithic (AS) blocks beyond one cluster: the split inversion over
        // the two field systems, float32 inverses
        int cq = 0, rq = 0;
        size_t smq = 0;
        const bool split = cx.variant == FSI_SMOOTHER_AS && !gj_tc_plan((int)D.max_block, &cq, &rq, &smq);
        if (split) {
            if (store != 1) {
                set_error("AS blocks of " + std::to_string(D.max_block) +
                          " dofs are inverted by the split method, which needs FSI_MIXED (float32 inverses)");
                return FSI_ERR_ARG;
            }
            FSI_TRY(launch_block_invert_schur(cx, D.A, D, H.off[3], method == FSI_FACTOR_TF32, cx.flags.as<int>(), s));
        } else if (method == FSI_FACTOR_FP64)
            FSI_TRY(launch_block_invert(D.A, D, store, cx.flags.as<int>(), s, cx.num_sms));
        else
            FSI_TRY(launch_block_invert_tc(D.A, D, store, method == FSI_FACTOR_TF32, cx.flags.as<int>(), s));
    }
    return FSI_OK;
}

fsi_status invert_level_blocks(Context &cx, Problem &pb, size_t l) {
    cudaStream_t s = cx.stream;
    FSI_CUDA(cudaMemsetAsync(cx.flags.p, 0, 16, s));
    FSI_TRY(launch_level_inversion(cx, pb, l, s));
    int fw[3] = {0, 0, 0};
    FSI_CUDA(cudaMemcpyAsync(fw, cx.flags.p, sizeof(fw), cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    if (fw[2]) {   // a bounded tensor-core wait of the factorisation gave up
        set_error("block factorisation on level " + std::to_string(l) + " timed out waiting for the tensor cores");
        return FSI_ERR_CUDA;
    }
    if (fw[0]) {
        set_error("a Schwarz block on level " + std::to_string(l) + " is singular");
        return FSI_ERR_ZERO_PIVOT;
    }
    return FSI_OK;
}

fsi_status setup_smoothers_problem(Context &cx, Problem &pb) {
    cudaStream_t s = cx.stream;
    if (cx.cascade) FSI_TRY(build_cascade(cx, pb));
    const bool mixed = cx.precision != FSI_FP64;             // float32 cycle
    const size_t tsz = mixed ? 4 : 8;
    const int store = cx.precision == FSI_MIXED_HALF ? 2 : (mixed ? 1 : 0);
    const int VW = store == 2 ? 8 : (store == 1 ? 4 : 2);   // 16-byte rows
    const size_t isz = store == 2 ? 2 : (store == 1 ? 4 : 8);
    for (size_t l = 0; l < pb.dev.size(); ++l) {
        LevelDev &D = pb.dev[l];
        LevelHost &H = pb.host[l];
        if (mixed) {
            FSI_TRY(make_f32(D.A, s));
            if (l >= 1) {
                FSI_TRY(make_f32(D.P, s));
                FSI_TRY(make_f32(D.R, s));
            }
            if (cx.cascade) {
                FSI_TRY(make_f32(D.Ac, s));
                if (l >= 1) FSI_TRY(make_f32(D.Rc, s));
            }
        }
        FSI_TRY(D.b.alloc((size_t)D.n * tsz));
        FSI_TRY(D.x.alloc((size_t)D.n * tsz));
        FSI_TRY(D.r.alloc((size_t)D.n * tsz));
        if (l == 0) continue;
        // locally multiplicative sweep on the cx.mult_levels finest levels
        const bool sweep = cx.variant == FSI_SMOOTHER_FS && cx.mult_levels > 0 &&
                           (int64_t)l + cx.mult_levels >= (int64_t)pb.dev.size();
        D.mult = sweep ? 1 : 0;
        D.mult_t_ready = false;
        D.passes.clear();
        std::vector<int32_t> tags, bpass;
        const bool fs = cx.variant == FSI_SMOOTHER_FS;
        build_blocks(H, pb.patch, D.h_blk_ptr, D.h_blk_idx, !fs, fs ? &tags : nullptr);
        D.n_blocks = (int64_t)D.h_blk_ptr.size() - 1;
        if (fs) sweep_passes(H, pb.patch, tags, bpass);
        if (sweep) {
            // blocks in sweep order: by pass (kind, colour), stable inside a pass
            std::vector<int64_t> ord(D.n_blocks);
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t c) { return bpass[a] < bpass[c]; });
            std::vector<int64_t> nptr(1, 0);
            std::vector<int32_t> nidx, npass;
            nidx.reserve(D.h_blk_idx.size());
            for (int64_t j : ord) {
                nidx.insert(nidx.end(), D.h_blk_idx.begin() + D.h_blk_ptr[j], D.h_blk_idx.begin() + D.h_blk_ptr[j + 1]);
                nptr.push_back((int64_t)nidx.size());
                npass.push_back(bpass[j]);
            }
            D.h_blk_ptr.swap(nptr);
            D.h_blk_idx.swap(nidx);
            bpass.swap(npass);
        }
        D.h_pass = bpass;                     // empty for AS blocks
        std::vector<int32_t> bp(D.h_blk_ptr.begin(), D.h_blk_ptr.end());
        std::vector<int64_t> off(D.n_blocks + 1, 0);
        std::vector<double> mult(D.n, 0.0);
        D.max_block = 0;
        for (int64_t j = 0; j < D.n_blocks; ++j) {
            const int64_t nj = D.h_blk_ptr[j + 1] - D.h_blk_ptr[j];
            D.max_block = std::max(D.max_block, nj);
            const int64_t ld = (nj + VW - 1) / VW * VW;
            off[j + 1] = off[j] + nj * ld;
            for (int64_t k = D.h_blk_ptr[j]; k < D.h_blk_ptr[j + 1]; ++k) mult[D.h_blk_idx[k]] += 1.0;
        }
        D.inv_elems = off[D.n_blocks];
        // partition-of-unity weights W_j = 1 / multiplicity (additive); the
        // multiplicative update formula adds each block's correction whole
        std::vector<double> w64(D.h_blk_idx.size());
        std::vector<float> w32(D.h_blk_idx.size());
        for (size_t k = 0; k < D.h_blk_idx.size(); ++k) {
            w64[k] = sweep ? 1.0 : 1.0 / mult[D.h_blk_idx[k]];
            w32[k] = (float)w64[k];
        }
        FSI_TRY(upload(D.blk_ptr, bp.data(), bp.size() * 4, s));
        FSI_TRY(upload(D.blk_idx, D.h_blk_idx.data(), D.h_blk_idx.size() * 4, s));
        FSI_TRY(upload(D.blk_off, off.data(), off.size() * 8, s));
        if (mixed) FSI_TRY(upload(D.blk_w, w32.data(), w32.size() * 4, s));
        else FSI_TRY(upload(D.blk_w, w64.data(), w64.size() * 8, s));
        // owners of the overlapping blocks (additive levels): the slots of every
        // covered dof in block order, for the owner-computes combination
        D.n_own = 0;
        if (!sweep) {
            const int64_t nnzb = (int64_t)D.h_blk_idx.size();
            std::vector<int32_t> ptr(D.n + 1, 0), pos(nnzb);
            for (int32_t i : D.h_blk_idx) ptr[i + 1]++;
            for (int64_t i = 0; i < D.n; ++i) ptr[i + 1] += ptr[i];
            std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
            for (int64_t k = 0; k < nnzb; ++k) pos[fill[D.h_blk_idx[k]]++] = (int32_t)k;
            std::vector<int32_t> odof, optr;
            std::vector<double> ow64;
            std::vector<float> ow32;
            for (int64_t i = 0; i < D.n; ++i) {
                if (ptr[i + 1] == ptr[i]) continue;
                odof.push_back((int32_t)i);
                optr.push_back(ptr[i]);
                ow64.push_back(1.0 / mult[i]);
                ow32.push_back((float)(1.0 / mult[i]));
            }
            optr.push_back((int32_t)nnzb);
            D.n_own = (int64_t)odof.size();
            if (D.n_own > 0) {
                FSI_TRY(upload(D.own_dof, odof.data(), odof.size() * 4, s));
                FSI_TRY(upload(D.own_ptr, optr.data(), optr.size() * 4, s));
                FSI_TRY(upload(D.own_pos, pos.data(), pos.size() * 4, s));
                if (mixed) FSI_TRY(upload(D.own_w, ow32.data(), ow32.size() * 4, s));
                else FSI_TRY(upload(D.own_w, ow64.data(), ow64.size() * 8, s));
                FSI_TRY(D.stage.alloc((size_t)nnzb * tsz));
            }
        }
        if (D.n_own == 0) {
            D.own_dof.release();
            D.own_ptr.release();
            D.own_pos.release();
            D.own_w.release();
            D.stage.release();
        }
        FSI_TRY(D.inv.alloc((size_t)D.inv_elems * isz));
        D.inv_store = store;
        if (store == 2) FSI_TRY(D.inv_scale.alloc(D.h_blk_idx.size() * 4));
        else D.inv_scale.release();
        // Jacobi rows: u^s (lumped K_u^s, Sec. 3.2) and fixed dofs
        std::vector<int32_t> jac;
        for (int64_t i = 0; i < D.n; ++i)
            if (H.fixed[i] || (cx.variant == FSI_SMOOTHER_FS && i >= H.off[3] && i < H.off[4]))
                jac.push_back((int32_t)i);
        D.n_jac = (int64_t)jac.size();
        FSI_TRY(upload(D.jac_idx, jac.data(), jac.size() * 4, s));
        FSI_TRY(D.jac_inv.alloc((size_t)std::max<int64_t>(D.n_jac, 1) * tsz));
        FSI_TRY(launch_jacobi_setup(D.A, D.jac_idx.as<int32_t>(), D.n_jac,
                                    mixed ? nullptr : D.jac_inv.as<double>(),
                                    mixed ? D.jac_inv.as<float>() : nullptr, s));
        // apply work items: whole blocks when there are enough of them to fill
        // the GPU, otherwise row chunks (multiples of 16 rows).  Splitting
        // blocks further (>= 64 items per SM) was measured slower on every
        // level it touched (128^2: 43 -> 52 us; 64^2: 17 -> 32 us): each chunk
        // gathers its block's residual again.
        {
            const int64_t want = 4 * (int64_t)cx.num_sms;
            const int64_t split = D.n_blocks >= want ? 1 : (want + D.n_blocks - 1) / D.n_blocks;
            std::vector<int32_t> it;
            std::vector<int64_t> pass_b0, pass_i0;    // sweep: first block and first item of every pass
            int64_t split_p = split;
            for (int64_t j = 0; j < D.n_blocks; ++j) {
                if (sweep && (j == 0 || bpass[j] != bpass[j - 1])) {
                    pass_b0.push_back(j);
                    pass_i0.push_back((int64_t)it.size() / 4);
                    // a pass is its own launch: split its blocks by rows until
                    // the pass alone gives every SM several items
                    int64_t nb = 0;
                    while (j + nb < D.n_blocks && bpass[j + nb] == bpass[j]) ++nb;
                    split_p = nb >= want ? 1 : (want + nb - 1) / nb;
                }
                const int nj = (int)(D.h_blk_ptr[j + 1] - D.h_blk_ptr[j]);
                int chunk = (int)((nj + split_p - 1) / split_p);
                chunk = std::max(16, (chunk + 15) / 16 * 16);
                for (int r0 = 0; r0 < nj; r0 += chunk) {
                    it.push_back((int32_t)j);
                    it.push_back(r0);
                    it.push_back(std::min(nj, r0 + chunk));
                    it.push_back(0);
                }
            }
            const int64_t blk_items = (int64_t)it.size() / 4;
            // Jacobi rows ride in the same launch: items (-1, k0, k1) over the jac list
            // (256 rows each: a sweep runs them as a pass of their own)
            for (int64_t k0 = 0; k0 < D.n_jac; k0 += 256) {
                it.push_back(-1);
                it.push_back((int32_t)k0);
                it.push_back((int32_t)std::min<int64_t>(D.n_jac, k0 + 256));
                it.push_back(0);
            }
            D.n_items = (int64_t)it.size() / 4;
            FSI_TRY(upload(D.items, it.data(), it.size() * 4, s));
            if (sweep) {
                int nc = 1;
                for (int a = 0; a < H.dim; ++a) nc *= colour_period(pb.patch);
                const size_t np = pass_b0.size();
                bool jac_placed = false;
                auto add_jacobi = [&]() {
                    if (jac_placed || D.n_jac == 0) return;
                    SweepPass P;
                    P.it0 = blk_items;
                    P.it1 = D.n_items;
                    P.field = 1;
                    P.jacobi = true;
                    P.rows = jac;
                    D.passes.push_back(std::move(P));
                    jac_placed = true;
                };
                for (size_t q = 0; q < np; ++q) {
                    const int64_t b0 = pass_b0[q], b1 = q + 1 < np ? pass_b0[q + 1] : D.n_blocks;
                    const int field = bpass[b0] / nc == 2 ? 1 : 0;
                    if (field == 1) add_jacobi();      // velocity field: K_u^s rows first
                    SweepPass P;
                    P.it0 = pass_i0[q];
                    P.it1 = q + 1 < np ? pass_i0[q + 1] : blk_items;
                    P.field = field;
                    P.rows.assign(D.h_blk_idx.begin() + D.h_blk_ptr[b0], D.h_blk_idx.begin() + D.h_blk_ptr[b1]);
                    std::sort(P.rows.begin(), P.rows.end());
                    D.passes.push_back(std::move(P));
                }
                add_jacobi();
                // free dofs of each field system of P2: 0 = d and p^s, 1 = u and p^f
                for (int f = 0; f < 2; ++f) {
                    D.h_keep[f].assign(D.n, 0);
                    for (int64_t i = 0; i < D.n; ++i)
                        D.h_keep[f][i] = (!H.fixed[i] && ((i < H.off[3]) == (f == 0))) ? 1 : 0;
                    FSI_TRY(upload(D.keep[f], D.h_keep[f].data(), (size_t)D.n, s));
                }
                for (auto &P : D.passes)
                    FSI_TRY(build_ell_subset(D.A, H.pattern, P.rows, D.h_keep[P.field], D.keep[P.field].as<uint8_t>(),
                                             P.ell, s, cx.probs.size() > 1));
                FSI_TRY(D.y.alloc((size_t)D.n * tsz));
                FSI_TRY(D.rr.alloc((size_t)D.n * tsz));
                FSI_CUDA(cudaMemsetAsync(D.y.p, 0, (size_t)D.n * tsz, s));
                FSI_CUDA(D.fj.create());
            } else {
                for (int f = 0; f < 2; ++f) {
                    D.h_keep[f].clear();
                    D.keep[f].release();
                }
                D.y.release();
                D.rr.release();
                D.fj.release();
            }
        }
        FSI_TRY(invert_level_blocks(cx, pb, l));
    }
    pb.transposes_ready = false;
    pb.m_alloc = 0;
    pb.ops_changed = false;
    pb.smoother_sig = smoother_signature(cx);
    drop_graphs(pb);
    return FSI_OK;
}

// New operator values with the smoother options and patterns of the last
// full set-up: refresh in place what derives from the values (float32
// copies, ELL values of the sweep passes, Jacobi rows, block inverses), so
// every buffer keeps its address and captured solve graphs stay valid.
// Anything else (first set-up, changed options, the swapped cascade, whose
// operators are rebuilt from the values) takes the full set-up.
fsi_status refactor_smoothers(Context &cx, Problem &pb) {
    if (pb.smoother_sig.empty() || pb.smoother_sig != smoother_signature(cx) || cx.cascade)
        return setup_smoothers_problem(cx, pb);
    cudaStream_t s = cx.stream;
    const bool mixed = cx.precision != FSI_FP64;
    for (size_t l = 0; l < pb.dev.size(); ++l) {
        LevelDev &D = pb.dev[l];
        if (mixed) FSI_TRY(make_f32(D.A, s));      // no-op when the float32 copy exists (kept current)
        if (l == 0) continue;
        FSI_TRY(launch_jacobi_setup(D.A, D.jac_idx.as<int32_t>(), D.n_jac, mixed ? nullptr : D.jac_inv.as<double>(),
                                    mixed ? D.jac_inv.as<float>() : nullptr, s));
        if (D.mult) {
            for (auto &P : D.passes)
                FSI_TRY(ell_subset_refill(D.A, P.ell, D.keep[P.field].as<uint8_t>(), s));
            D.mult_t_ready = false;
        }
        FSI_TRY(invert_level_blocks(cx, pb, l));
    }
    pb.transposes_ready = false;
    pb.ops_changed = false;
    return FSI_OK;
}

template <class T>
fsi_status apply_smoother_t(Context &cx, LevelDev &L, const double *r, double *y, int tr) {
    cudaStream_t s = cx.stream;
    DevBuf rt, yt;
    FSI_TRY(rt.alloc((size_t)L.n * sizeof(T)));
    FSI_TRY(yt.alloc((size_t)L.n * sizeof(T)));
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f64_f32(r, rt.as<float>(), L.n, s));
    else FSI_CUDA(cudaMemcpyAsync(rt.p, r, (size_t)L.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaMemsetAsync(yt.p, 0, (size_t)L.n * sizeof(T), s));
    const double om = cx.omega;
    cx.omega = 1.0;   // plain P2^{-1} r
    fsi_status st = smooth_apply<T>(cx, L, rt.as<T>(), yt.as<T>(), tr != 0);
    cx.omega = om;
    FSI_TRY(st);
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f32_f64(yt.as<float>(), y, L.n, s));
    else FSI_CUDA(cudaMemcpyAsync(y, yt.p, (size_t)L.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

template <class T>
fsi_status apply_vcycle_t(Context &cx, Problem &pb, const double *v, double *z, int tr) {
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    DevBuf &bt = F.b, &xt = F.x;     // the fine cycle vectors, as inside a solve
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f64_f32(v, bt.as<float>(), F.n, s));
    else FSI_CUDA(cudaMemcpyAsync(bt.p, v, (size_t)F.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_TRY(vcycle<T>(cx, pb, (int)pb.dev.size() - 1, bt.as<T>(), xt.as<T>(), tr != 0));
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f32_f64(xt.as<float>(), z, F.n, s));
    else FSI_CUDA(cudaMemcpyAsync(z, xt.p, (size_t)F.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

Problem *get_prob(const fsi_ctx *ctx, int prob, int level) {
    const Context *cx = reinterpret_cast<const Context *>(ctx);
    if (!cx || prob < 0 || prob >= (int)cx->probs.size()) return nullptr;
    Problem *pb = const_cast<Problem *>(&cx->probs[prob]);
    if (level < 0 || level >= (int)pb->dev.size()) return nullptr;
    return pb;
}

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" {

const char *fsi_last_error(void) { return g_last_error.c_str(); }

fsi_status fsi_setup_hierarchy(const fsi_problem *probs, int n_probs, const fsi_hier_opts *opts,
                               void *cuda_stream, fsi_ctx **out) {
    g_last_error.clear();
    if (!probs || n_probs < 1 || !out) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    *out = nullptr;
    std::unique_ptr<Context> cx(new Context());
    FSI_CUDA(cudaGetDevice(&cx->device));
    cx->stream = static_cast<cudaStream_t>(cuda_stream);
    cx->restriction = opts ? opts->restriction : 0;
    if (cx->restriction != 0 && cx->restriction != 1) { set_error("restriction must be 0 or 1"); return FSI_ERR_ARG; }
    cx->nonlinear = opts ? opts->nonlinear : 0;
    if (cx->nonlinear != 0 && cx->nonlinear != 1) { set_error("nonlinear must be 0 or 1"); return FSI_ERR_ARG; }
    FSI_CUDA(cudaDeviceGetAttribute(&cx->num_sms, cudaDevAttrMultiProcessorCount, cx->device));
    FSI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&cx->h_pinned), 64 * 8));
    FSI_CUDA(cudaStreamCreateWithFlags(&cx->work, cudaStreamNonBlocking));
    FSI_CUDA(cudaEventCreateWithFlags(&cx->ev_in, cudaEventDisableTiming));
    FSI_CUDA(cudaEventCreateWithFlags(&cx->ev_out, cudaEventDisableTiming));
    {
        const char *g = getenv("FSI_USE_GRAPHS");
        cx->use_graphs = !(g && g[0] == '0');
        const char *dl = getenv("FSI_DEVICE_LOOP");
        cx->device_loop = !(dl && dl[0] == '0');
    }
    for (auto &c : cx->cap) FSI_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    FSI_TRY(cx->flags.alloc(16));
    cx->probs.resize(n_probs);
    for (int i = 0; i < n_probs; ++i) {
        fsi_status st = setup_problem(*cx, cx->probs[i], probs[i]);
        if (st != FSI_OK) {
            cudaFreeHost(cx->h_pinned);
            cx->h_pinned = nullptr;
            return st;
        }
    }
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    *out = reinterpret_cast<fsi_ctx *>(cx.release());
    return FSI_OK;
}

fsi_status fsi_setup_host_only(const fsi_problem *prob, const fsi_hier_opts *opts, int patch, fsi_ctx **out) {
    g_last_error.clear();
    if (!prob || !out || patch < 0 || patch > 16) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    *out = nullptr;
    std::unique_ptr<Context> cx(new Context());
    cx->host_only = true;
    cx->patch = patch;
    cx->restriction = opts ? opts->restriction : 0;
    if (cx->restriction != 0 && cx->restriction != 1) { set_error("restriction must be 0 or 1"); return FSI_ERR_ARG; }
    cx->nonlinear = opts ? opts->nonlinear : 0;
    if (cx->nonlinear != 0 && cx->nonlinear != 1) { set_error("nonlinear must be 0 or 1"); return FSI_ERR_ARG; }
    cx->probs.resize(1);
    FSI_TRY(setup_problem(*cx, cx->probs[0], *prob));
    *out = reinterpret_cast<fsi_ctx *>(cx.release());
    return FSI_OK;
}

fsi_status fsi_get_pattern(const fsi_ctx *ctx, int prob, int level, int64_t *row_ptr, int32_t *col) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || !row_ptr || !col) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const HostCSR &P = pb->host[level].pattern;
    std::memcpy(row_ptr, P.ptr.data(), P.ptr.size() * 8);
    std::memcpy(col, P.col.data(), P.col.size() * 4);
    return FSI_OK;
}

fsi_status fsi_setup_smoothers(fsi_ctx *ctx, const fsi_smoother_opts *opts) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !opts) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (opts->precision < FSI_FP64 || opts->precision > FSI_MIXED_HALF || opts->patch < 1 || opts->patch > 16 ||
        !(opts->omega > 0) || opts->nu_pre < 1 || opts->nu_post < 1 || opts->nu_pre > 8 || opts->nu_post > 8 ||
        opts->factor < FSI_FACTOR_AUTO || opts->factor > FSI_FACTOR_TF32 ||
        (opts->variant != FSI_SMOOTHER_FS && opts->variant != FSI_SMOOTHER_AS) ||
        opts->mult_levels < 0 ||
        (opts->mult_levels > 0 && opts->variant != FSI_SMOOTHER_FS) ||
        (opts->cascade != 0 && opts->cascade != 1) ||
        (opts->cascade == 1 && opts->variant != FSI_SMOOTHER_FS)) {
        set_error("smoother options out of range");
        return FSI_ERR_ARG;
    }
    if (opts->precision == FSI_FP64 && opts->factor >= FSI_FACTOR_FP32) {
        set_error("float32 block inversion needs a mixed precision");
        return FSI_ERR_ARG;
    }
    DeviceGuard guard(cx->device);
    cx->precision = opts->precision;
    cx->patch = opts->patch;
    for (auto &pb : cx->probs) pb.patch = opts->patch;
    cx->omega = opts->omega;
    cx->nu_pre = opts->nu_pre;
    cx->nu_post = opts->nu_post;
    cx->factor = opts->factor;
    cx->variant = opts->variant;
    cx->mult_levels = opts->mult_levels;
    cx->cascade = opts->cascade;
    cx->smoothers_ready = false;
    for (auto &pb : cx->probs) FSI_TRY(setup_smoothers_problem(*cx, pb));
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    if (!cx->ev_marks.empty()) collect_marks(*cx);
    cx->smoothers_ready = true;
    cx->smoothers_configured = true;
    return FSI_OK;
}

}  // extern "C"

namespace fsi {
namespace {

// ------------------------------------------------- device-driven FGMRES
// The whole solve as one CUDA graph: the prologue (||b||, r0 = b - A x0,
// ||r0||) is followed by a WHILE node over restart cycles whose body starts
// the basis, runs a nested WHILE node over Arnoldi steps, and ends with
// x += Z y and the float64 true residual.  The loop conditions are set on
// the device (fg_start / givens / fg_cycle kernels), so a solve needs no
// host round trip; the host reads the control block once at the end.  b and
// x live in fixed per-problem buffers so the graph is captured once per
// direction and restart length and replayed for any caller pointers.

// one Arnoldi step with the column index on the device (loop body):
// z_j = M^{-1} v_j and w = A z_j, then a SWITCH node whose case c holds the
// Gram-Schmidt/Givens kernels instantiated for nv <= nv_class_bound(c)
// (the case is chosen on the device from fg->k by take_column), so early
// steps keep the small-register variants instead of the widest one.
template <class T>
fsi_status issue_step_dev_head(Context &cx, Problem &pb, bool tr, cudaGraphConditionalHandle sel) {
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    const int L = (int)pb.dev.size();
    const DevCSR &A = tr ? F.AT : F.A;
    FgState *fg = pb.fg.as<FgState>();
    double *V = pb.V.as<double>(), *w = pb.w.as<double>(), *Z = pb.Z.as<double>();
    double *zf = pb.zbuf.as<double>();
    FSI_TRY(launch_take_column<double, T>(V, n, fg, F.b.as<T>(), n, s, sel, F.x.as<T>()));
    FSI_TRY(vcycle<T>(cx, pb, L - 1, F.b.as<T>(), F.x.as<T>(), tr, true));   // x zeroed above
    PdlScope pdl;                     // both follow a kernel of the cycle
    FSI_TRY(launch_store_column<T>(F.x.as<T>(), zf, Z, n, fg, n, s));
    FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), zf, (const double *)nullptr, w, SPMV_SET, s));
    return FSI_OK;
}

fsi_status issue_step_dev_tail(Context &cx, Problem &pb, int m, int nv_bound, cudaGraphConditionalHandle loop) {
    cudaStream_t s = cx.stream;
    const int64_t n = pb.dev.back().n;
    FgState *fg = pb.fg.as<FgState>();
    double *V = pb.V.as<double>(), *H = pb.H.as<double>(), *g = pb.g.as<double>();
    double *w = pb.w.as<double>(), *scal = pb.scal.as<double>();
    double *part = pb.partials.as<double>(), *h1 = pb.h1.as<double>(), *h2 = pb.h2.as<double>();
    float *V32 = cx.precision != FSI_FP64 ? pb.V32.as<float>() : nullptr;
    if (V32) FSI_TRY(launch_mdot32(V32, n, nv_bound, w, n, part, NDOT, s, fg));
    else FSI_TRY(launch_mdot(V, n, nv_bound, w, n, part, NDOT, s, fg));
    PdlScope pdl;                     // the rest of the step follows kernels of this body
    FSI_TRY(launch_reduce_partials(part, NDOT, nv_bound, h1, 0, s, fg));
    FSI_TRY(launch_update_dot(w, V, n, nv_bound, h1, n, part, NRED, 0, s, fg, V32));
    FSI_TRY(launch_reduce_partials(part, NRED, nv_bound, h2, 0, s, fg));
    FSI_TRY(launch_update_dot(w, V, n, nv_bound, h2, n, part, NRED, 1, s, fg));
    FSI_TRY(launch_reduce_partials(part, NRED, 1, scal + 7, 0, s));
    FSI_TRY(launch_givens(H, m + 1, 0, h1, h2, scal + 7, pb.cs.as<double>(), pb.sn.as<double>(), g, scal, s, fg,
                          loop));
    FSI_TRY(launch_scale_copy(w, V, scal, 1, n, s, fg, n, V32));
    return FSI_OK;
}

// append a conditional node (WHILE or SWITCH with `size` cases) at the
// capture position of stream s; returns its body graphs
fsi_status add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                           unsigned size, cudaGraphNode_t *node, cudaGraph_t *bodies) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    FSI_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) { set_error("stream is not capturing"); return FSI_ERR_STATE; }
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    FSI_CUDA(cudaGraphAddNode(node, g, deps, nullptr, nd, &p));
    for (unsigned i = 0; i < size; ++i) bodies[i] = p.conditional.phGraph_out[i];
    FSI_CUDA(cudaStreamUpdateCaptureDependencies(s, node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return FSI_OK;
}

// One problem's whole solve captured into `top` as a chain with no
// dependencies (a root of the graph); cnt_out: kernels in the prologue, per
// restart cycle outside the steps, per Arnoldi step.
template <class T>
fsi_status capture_chain(Context &cx, Problem &pb, bool tr, int m, cudaGraph_t top, int64_t cnt_out[3]) {
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    const DevCSR &A = tr ? F.AT : F.A;
    FgState *fg = pb.fg.as<FgState>();
    double *scal = pb.scal.as<double>(), *r = pb.rvec.as<double>();
    double *b = pb.bbuf.as<double>(), *x = pb.xbuf.as<double>();
    cudaStream_t s0 = pb.stream, s1 = cx.cap[0], s2 = cx.cap[1], s3 = cx.cap[2];
    cudaStream_t saved = cx.stream;
    int64_t cnt[3] = {0, 0, 0};
    fsi_status st = FSI_OK;
    int capturing = 0;        // streams in capture, innermost last
    cudaStream_t active[4] = {s0, s1, s2, s3};
    auto fail = [&](fsi_status e) {
        // captures into existing graphs: the bodies belong to their nodes
        for (int i = capturing - 1; i >= 0; --i) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(active[i], &junk);
        }
        cudaGetLastError();
        cx.stream = saved;
        return e;
    };
#define FSI_CAP(...)                                   \
    do {                                               \
        st = (__VA_ARGS__);                            \
        if (st != FSI_OK) return fail(st);             \
    } while (0)
#define FSI_CAPCUDA(...)                               \
    do {                                               \
        cudaError_t e_ = (__VA_ARGS__);                \
        if (e_ != cudaSuccess) {                       \
            set_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
            return fail(FSI_ERR_CUDA);                 \
        }                                              \
    } while (0)
    const int64_t c0 = launches_so_far();
    cudaGraphConditionalHandle h_out = 0, h_in = 0;
    FSI_CAPCUDA(cudaGraphConditionalHandleCreate(&h_out, top, 0, cudaGraphCondAssignDefault));
    // prologue
    FSI_CAPCUDA(cudaStreamBeginCaptureToGraph(s0, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = 1;
    cx.stream = s0;
    FSI_CAP(norm2(cx, pb, b, n, 5));
    FSI_CAP(launch_spmv<double, double, double>(A, A.val64.as<double>(), x, b, r, SPMV_RESID, s0));
    FSI_CAP(norm2(cx, pb, r, n, 6));
    FSI_CAP(launch_fg_start(scal, fg, h_out, s0));
    const int64_t c1 = launches_so_far();
    // outer loop over restart cycles
    cudaGraphNode_t w_out = nullptr, w_in = nullptr;
    cudaGraph_t body_out = nullptr, body_in = nullptr;
    FSI_CAP(add_conditional(s0, h_out, cudaGraphCondTypeWhile, 1, &w_out, &body_out));
    FSI_CAPCUDA(cudaGraphConditionalHandleCreate(&h_in, body_out, 0, 0));
    FSI_CAPCUDA(cudaStreamBeginCaptureToGraph(s1, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = 2;
    cx.stream = s1;
    FSI_CAP(launch_init_basis(r, pb.V.as<double>(), pb.g.as<double>(), m, scal + 6, n, s1, fg, h_in,
                              cx.precision != FSI_FP64 ? pb.V32.as<float>() : nullptr));
    FSI_CAP(add_conditional(s1, h_in, cudaGraphCondTypeWhile, 1, &w_in, &body_in));
    // inner loop: Arnoldi steps
    const int64_t c2 = launches_so_far();
    FSI_CAPCUDA(cudaStreamBeginCaptureToGraph(s2, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = 3;
    cx.stream = s2;
    cudaGraphConditionalHandle h_sel = 0;
    FSI_CAPCUDA(cudaGraphConditionalHandleCreate(&h_sel, body_in, 0, 0));
    FSI_CAP(issue_step_dev_head<T>(cx, pb, tr, h_sel));
    int ncls = 1;
    while (ncls < NV_CLASSES && nv_class_bound(ncls - 1) < m) ++ncls;    // cases covering nv <= m
    cudaGraphNode_t w_sel = nullptr;
    cudaGraph_t cases[NV_CLASSES] = {};
    FSI_CAP(add_conditional(s2, h_sel, cudaGraphCondTypeSwitch, (unsigned)ncls, &w_sel, cases));
    int64_t tail_kernels = 0;
    for (int c = 0; c < ncls; ++c) {
        const int64_t t0 = launches_so_far();
        FSI_CAPCUDA(cudaStreamBeginCaptureToGraph(s3, cases[c], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capturing = 4;
        cx.stream = s3;
        FSI_CAP(issue_step_dev_tail(cx, pb, m, std::min(nv_class_bound(c), m), h_in));
        cudaGraph_t g3 = nullptr;
        FSI_CAPCUDA(cudaStreamEndCapture(s3, &g3));
        capturing = 3;
        tail_kernels = launches_so_far() - t0;     // the same count in every case
    }
    cx.stream = s2;
    {
        cudaGraph_t g2 = nullptr;
        FSI_CAPCUDA(cudaStreamEndCapture(s2, &g2));
        capturing = 2;
    }
    const int64_t c3 = launches_so_far();
    // end of a cycle: x += Z y, true residual, restart test
    cx.stream = s1;
    FSI_CAP(launch_backsolve(pb.H.as<double>(), m + 1, 0, pb.g.as<double>(), pb.y.as<double>(), s1, fg));
    FSI_CAP(launch_combine<double>(x, pb.Z.as<double>(), n, 0, pb.y.as<double>(), n, s1, fg));
    FSI_CAP(launch_spmv<double, double, double>(A, A.val64.as<double>(), x, b, r, SPMV_RESID, s1));
    FSI_CAP(norm2(cx, pb, r, n, 6));
    FSI_CAP(launch_fg_cycle(scal, fg, h_out, s1));
    {
        cudaGraph_t g1 = nullptr;
        FSI_CAPCUDA(cudaStreamEndCapture(s1, &g1));
        capturing = 1;
    }
    const int64_t c4 = launches_so_far();
    {
        cudaGraph_t g0 = nullptr;
        FSI_CAPCUDA(cudaStreamEndCapture(s0, &g0));
        capturing = 0;
    }
    cx.stream = saved;
#undef FSI_CAP
#undef FSI_CAPCUDA
    cnt[0] = c1 - c0;                       // prologue
    cnt[1] = (c2 - c1) + (c4 - c3);         // per cycle, outside the steps
    cnt[2] = (c3 - c2) - (int64_t)(ncls - 1) * tail_kernels;   // per Arnoldi step (one case runs)
    count_launch(-(int)(c4 - c0));          // captured, not run
    for (int i = 0; i < 3; ++i) cnt_out[i] = cnt[i];
    (void)cnt;
    return FSI_OK;
}

template <class T>
fsi_status capture_solve(Context &cx, Problem &pb, bool tr, int m) {
    cudaGraph_t top = nullptr;
    FSI_CUDA(cudaGraphCreate(&top, 0));
    int64_t cnt[3] = {0, 0, 0};
    fsi_status st = capture_chain<T>(cx, pb, tr, m, top, cnt);
    cudaGraphExec_t exec = nullptr;
    if (st == FSI_OK && cudaGraphInstantiate(&exec, top, 0) != cudaSuccess) {
        set_error("cudaGraphInstantiate of the solve graph failed");
        st = FSI_ERR_CUDA;
    }
    cudaGraphDestroy(top);
    FSI_TRY(st);
    const int d = tr ? 1 : 0;
    if (pb.solve_graph[d]) cudaGraphExecDestroy(pb.solve_graph[d]);
    pb.solve_graph[d] = exec;
    pb.solve_graph_m[d] = m;
    for (int i = 0; i < 3; ++i) pb.graph_counts[d][i] = cnt[i];
    return FSI_OK;
}

// Every problem of a batch in one graph: one root chain per problem (its
// prologue and restart/Arnoldi WHILE loops, conditions on its own control
// block), so one launch solves all systems and each stops on its own test.
template <class T>
fsi_status capture_batch(Context &cx, bool tr, int m) {
    cudaGraph_t top = nullptr;
    FSI_CUDA(cudaGraphCreate(&top, 0));
    const int d = tr ? 1 : 0;
    fsi_status st = FSI_OK;
    for (auto &pb : cx.probs) {
        int64_t cnt[3] = {0, 0, 0};
        st = capture_chain<T>(cx, pb, tr, m, top, cnt);
        if (st != FSI_OK) break;
        for (int i = 0; i < 3; ++i) pb.graph_counts[d][i] = cnt[i];
    }
    cudaGraphExec_t exec = nullptr;
    if (st == FSI_OK && cudaGraphInstantiate(&exec, top, 0) != cudaSuccess) {
        set_error("cudaGraphInstantiate of the batch graph failed");
        st = FSI_ERR_CUDA;
    }
    cudaGraphDestroy(top);
    FSI_TRY(st);
    if (cx.batch_graph[d]) cudaGraphExecDestroy(cx.batch_graph[d]);
    cx.batch_graph[d] = exec;
    cx.batch_graph_m[d] = m;
    cx.batch_epoch[d] = g_graph_epoch.load();
    return FSI_OK;
}

template <class T>
fsi_status run_device_loop(Context &cx, std::vector<Run> &runs) {
    cudaStream_t user = cx.stream;
    FSI_CUDA(cudaMemsetAsync(cx.flags.as<int>() + 2, 0, 4, user));   // kernel error word
    FSI_CUDA(cudaEventRecord(cx.ev_in, user));
    // a batch over every problem of the context in one graph
    const bool batch = runs.size() > 1 && runs.size() == cx.probs.size();
    const int bd = runs[0].tr ? 1 : 0, bm = runs[0].o.restart;
    if (batch) {
        for (auto &R : runs) {
            Problem &pb = *R.pb;
            FSI_TRY(ensure_workspace(cx, pb, bm));
            if (!pb.bbuf.p) {
                const int64_t n = pb.dev.back().n;
                FSI_TRY(pb.bbuf.alloc((size_t)n * 8));
                FSI_TRY(pb.xbuf.alloc((size_t)n * 8));
                FSI_TRY(pb.zbuf.alloc((size_t)n * 8));
            }
        }
        if (!cx.batch_graph[bd] || cx.batch_graph_m[bd] != bm || cx.batch_epoch[bd] != g_graph_epoch.load())
            FSI_TRY(capture_batch<T>(cx, runs[0].tr, bm));
    }
    for (auto &R : runs) {
        Problem &pb = *R.pb;
        const int m = R.o.restart;
        const int d = R.tr ? 1 : 0;
        const int64_t n = pb.dev.back().n;
        if (!batch) {
            FSI_TRY(ensure_workspace(cx, pb, m));
            if (!pb.bbuf.p) {
                FSI_TRY(pb.bbuf.alloc((size_t)n * 8));
                FSI_TRY(pb.xbuf.alloc((size_t)n * 8));
                FSI_TRY(pb.zbuf.alloc((size_t)n * 8));
            }
            FSI_CUDA(cudaStreamWaitEvent(pb.stream, cx.ev_in, 0));
            if (!pb.solve_graph[d] || pb.solve_graph_m[d] != m) FSI_TRY(capture_solve<T>(cx, pb, R.tr, m));
        }
        R.st = fsi_solve_stats();
        FgState &in = pb.h_fg[0];
        in = FgState();
        in.rtol = R.o.rtol;
        in.max_iters = R.o.max_iters;
        in.m = m;
        cudaStream_t s = batch ? user : pb.stream;
        if (!batch) FSI_CUDA(cudaEventRecord(pb.ev_a, s));
        FSI_CUDA(cudaMemcpyAsync(pb.fg.p, &in, sizeof(FgState), cudaMemcpyHostToDevice, s));
        FSI_CUDA(cudaMemcpyAsync(pb.bbuf.p, R.b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        if (R.o.use_x0) FSI_CUDA(cudaMemcpyAsync(pb.xbuf.p, R.x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        else FSI_CUDA(cudaMemsetAsync(pb.xbuf.p, 0, (size_t)n * 8, s));
        if (batch) continue;
        FSI_CUDA(cudaGraphLaunch(pb.solve_graph[d], s));
        FSI_CUDA(cudaMemcpyAsync(R.x, pb.xbuf.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        FSI_CUDA(cudaMemcpyAsync(&pb.h_fg[1], pb.fg.p, sizeof(FgState), cudaMemcpyDeviceToHost, s));
        FSI_CUDA(cudaEventRecord(pb.ev_b, s));
    }
    if (batch) {
        // one launch for every system; each chain stops on its own test
        Problem &p0 = *runs[0].pb;
        FSI_CUDA(cudaEventRecord(p0.ev_a, user));
        FSI_CUDA(cudaGraphLaunch(cx.batch_graph[bd], user));
        FSI_CUDA(cudaEventRecord(p0.ev_b, user));
        for (auto &R : runs) {
            Problem &pb = *R.pb;
            FSI_CUDA(cudaMemcpyAsync(R.x, pb.xbuf.p, (size_t)pb.dev.back().n * 8, cudaMemcpyDeviceToDevice, user));
            FSI_CUDA(cudaMemcpyAsync(&pb.h_fg[1], pb.fg.p, sizeof(FgState), cudaMemcpyDeviceToHost, user));
        }
        FSI_CUDA(cudaStreamSynchronize(user));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p0.ev_a, p0.ev_b);
        batch_ms_last = ms;
    }
    fsi_status err = FSI_OK;
    for (auto &R : runs) {
        Problem &pb = *R.pb;
        cudaError_t ce = cudaStreamSynchronize(pb.stream);
        if (ce != cudaSuccess) {
            set_error(std::string("solve stream: ") + cudaGetErrorString(ce));
            err = FSI_ERR_CUDA;
            continue;
        }
        const FgState &o = pb.h_fg[1];
        const int d = R.tr ? 1 : 0;
        count_launch((int)(pb.graph_counts[d][0] + o.cycles * pb.graph_counts[d][1] +
                           o.its * pb.graph_counts[d][2]));
        R.its = o.its;
        R.bnorm = o.bnorm;
        R.beta = o.beta;
        R.st.r0 = o.r0;
        R.st.cycles = o.cycles;
        fsi_status status = FSI_OK;
        if (!std::isfinite(o.bnorm)) {
            set_error("right-hand side has a non-finite norm");
            R.beta = NAN;
            status = FSI_ERR_NONFINITE;
        } else if (o.bnorm == 0.0) {
            FSI_CUDA(cudaMemsetAsync(R.x, 0, (size_t)pb.dev.back().n * 8, pb.stream));
            R.beta = 0.0;
        } else if (o.flags & 1) {
            set_error("non-finite value in the Arnoldi process");
            R.beta = NAN;
            status = FSI_ERR_NONFINITE;
        }
        finish(R, status);
        float ms = 0.f;
        if (batch) R.st.solve_ms = batch_ms_last;
        else if (cudaEventElapsedTime(&ms, pb.ev_a, pb.ev_b) == cudaSuccess) R.st.solve_ms = ms;
    }
    for (auto &R : runs) {
        FSI_CUDA(cudaEventRecord(cx.ev_out, R.pb->stream));
        FSI_CUDA(cudaStreamWaitEvent(user, cx.ev_out, 0));
    }
    return err;
}

}  // namespace
}  // namespace fsi

namespace fsi {
namespace {
// Algorithmic bytes (the data the method must move) of one smoothing step on
// level L: every block's inverse (n^2 entries) with its index, weight,
// gathered residual and updated correction entries (+ a float32 row scale
// with FP16 storage), the Jacobi rows; a multiplicative sweep adds the pass
// residuals r - A_FF y on the rows of every pass but the first of each field
// (A_FF entries with their column indices; permutation index, b, y and rr
// per row) and the closing x += omega y with y cleared.
double smoother_bytes(const Context &cx, const LevelDev &L) {
    const double ts = cx.precision != FSI_FP64 ? 4.0 : 8.0;
    const double is = cx.precision == FSI_MIXED_HALF ? 2.0 : ts;
    const double rowx = cx.precision == FSI_MIXED_HALF ? 4.0 : 0.0;
    double b = 0.0;
    for (int64_t j = 0; j + 1 < (int64_t)L.h_blk_ptr.size(); ++j) {
        const double nj = (double)(L.h_blk_ptr[j + 1] - L.h_blk_ptr[j]);
        b += nj * nj * is + nj * (4.0 + ts + ts + 2.0 * ts + rowx);
    }
    b += (double)L.n_jac * (4.0 + ts + ts + 2.0 * ts);
    if (L.mult) {
        bool started[2] = {false, false};
        for (const auto &P : L.passes) {
            if (started[P.field]) b += (double)P.ell.nnz * (ts + 4.0) + (double)P.rows.size() * (4.0 + 3.0 * ts);
            started[P.field] = true;
        }
        b += (double)L.n * 4.0 * ts;
    }
    return b;
}

// one sparse product y = b - A x (or A x): values and column indices, row
// pointers, x, b and y
double spmv_bytes(const DevCSR &A, double ts) {
    return (double)A.nnz * (ts + 4.0) + (double)(A.n_rows + 1) * 4.0 + (double)A.n_rows * 3.0 * ts;
}

// one V-cycle from a zero guess on the fine level (Sec. 3.2): per level l >= 1
// two smoothing steps, two residuals (before restriction, before the
// post-smoothing step), restriction and prolongation; the coarse inverse
// GEMV; the fine-level casts of v and z in the mixed modes
double cycle_bytes(const Context &cx, const Problem &pb) {
    const double ts = cx.precision != FSI_FP64 ? 4.0 : 8.0;
    double b = (double)pb.n0 * (double)pb.n0 * 8.0 + (double)pb.n0 * 2.0 * ts;
    for (size_t l = 1; l < pb.dev.size(); ++l) {
        const LevelDev &L = pb.dev[l];
        const DevCSR &A = cx.cascade ? L.Ac : L.A;
        const DevCSR &R = cx.cascade ? L.Rc : L.R;
        b += 2.0 * smoother_bytes(cx, L) + 2.0 * spmv_bytes(A, ts) + spmv_bytes(R, ts) + spmv_bytes(L.P, ts);
    }
    if (cx.precision != FSI_FP64) b += (double)pb.dev.back().n * 2.0 * 12.0;
    return b;
}
}  // namespace
}  // namespace fsi

extern "C" {

// Hardware work queues of the context (CUDA_DEVICE_MAX_CONNECTIONS, default
// 8).  Streams beyond that share queues, and a whole-solve graph then blocks
// every solve queued behind it, so partial batches larger than this advance
// in host-driven rounds of one Arnoldi step instead.  A batch over every
// problem of the context is one graph launch (capture_batch).
static int hw_queues() {
    const char *e = getenv("CUDA_DEVICE_MAX_CONNECTIONS");
    const int v = e ? atoi(e) : 0;
    return v > 0 ? v : 8;
}

static fsi_status solve_runs(Context &cx, std::vector<Run> &runs) {
    const bool whole = runs.size() > 1 && runs.size() == cx.probs.size();
    const bool dev_loop = cx.use_graphs && cx.device_loop && !cx.profile &&
                          ((int)runs.size() <= hw_queues() || whole);
    fsi_status s = dev_loop ? ((cx.precision != FSI_FP64) ? run_device_loop<float>(cx, runs)
                                                          : run_device_loop<double>(cx, runs))
                            : ((cx.precision != FSI_FP64) ? run_batch<float>(cx, runs) : run_batch<double>(cx, runs));
    if (s != FSI_OK) return s;
    fsi_status worst = FSI_OK;
    for (auto &R : runs)
        if (R.status != FSI_OK && worst == FSI_OK) worst = R.status;
    return worst;
}

static fsi_status solve_one(Context &cx, Problem &pb, const double *b, double *x, const fsi_solve_opts *o,
                            fsi_solve_stats *st, bool tr) {
    std::vector<Run> runs(1);
    runs[0].pb = &pb;
    runs[0].b = b;
    runs[0].x = x;
    runs[0].tr = tr;
    runs[0].o = *o;
    fsi_status s = solve_runs(cx, runs);
    if (st) *st = runs[0].st;
    return s;
}

fsi_status fsi_solve(fsi_ctx *ctx, const double *b, double *x, const fsi_solve_opts *opts, fsi_solve_stats *st) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !b || !x) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    FSI_TRY(check_opts(opts));
    if (!cx->smoothers_ready) { set_error("fsi_setup_smoothers has not completed"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    return solve_one(*cx, cx->probs[0], b, x, opts, st, false);
}

fsi_status fsi_solve_batched(fsi_ctx *ctx, const double *const *b, double *const *x, const fsi_solve_opts *opts,
                             fsi_solve_stats *st) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !b || !x) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    FSI_TRY(check_opts(opts));
    if (!cx->smoothers_ready) { set_error("fsi_setup_smoothers has not completed"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    std::vector<Run> runs(cx->probs.size());
    for (size_t i = 0; i < cx->probs.size(); ++i) {
        if (!b[i] || !x[i]) { set_error("NULL vector in batch"); return FSI_ERR_ARG; }
        runs[i].pb = &cx->probs[i];
        runs[i].b = b[i];
        runs[i].x = x[i];
        runs[i].o = *opts;
    }
    fsi_status s = solve_runs(*cx, runs);
    if (st)
        for (size_t i = 0; i < runs.size(); ++i) st[i] = runs[i].st;
    return s;
}

fsi_status fsi_adjoint(fsi_ctx *ctx, const double *w, const double *x, double *lambda, double *dA_vals,
                       double *dmu_s, const fsi_solve_opts *opts, fsi_solve_stats *st) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !w || !x || !lambda) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    FSI_TRY(check_opts(opts));
    if (!cx->smoothers_ready) { set_error("fsi_setup_smoothers has not completed"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    Problem &pb = cx->probs[0];
    FSI_TRY(build_transposes(*cx, pb));
    fsi_status s = solve_one(*cx, pb, w, lambda, opts, st, true);
    if (s != FSI_OK && s != FSI_ERR_NOT_CONVERGED) return s;
    LevelDev &F = pb.dev.back();
    if (dA_vals) FSI_TRY(launch_pattern_grad(F.A, lambda, x, dA_vals, cx->stream));
    if (dmu_s && !pb.dA_mu.p) {
        set_error("dJ/dmu_s is not available: the operator is a Jacobian of the nonlinear residual");
        return FSI_ERR_STATE;
    }
    if (dmu_s) {
        // -lambda^T (dA/dmu_s) x
        FSI_TRY(launch_spmv<double, double, double>(F.A, pb.dA_mu.as<double>(), x, (const double *)nullptr,
                                                    pb.w.as<double>(), SPMV_SET, cx->stream));
        FSI_TRY(launch_mdot(lambda, F.n, 1, pb.w.as<double>(), F.n, pb.partials.as<double>(), NRED, cx->stream));
        FSI_TRY(launch_reduce_partials(pb.partials.as<double>(), NRED, 1, pb.scal.as<double>() + 8, 0, cx->stream));
        FSI_CUDA(cudaMemcpyAsync(cx->h_pinned, pb.scal.as<double>() + 8, 8, cudaMemcpyDeviceToHost, cx->stream));
        FSI_CUDA(cudaStreamSynchronize(cx->stream));
        *dmu_s = -reinterpret_cast<const double *>(cx->h_pinned)[0];
    }
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    return s;
}

fsi_status fsi_profile(fsi_ctx *ctx, int mode, double *out) {
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !out || mode < 0 || mode > 3) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    double fp64_gflops = 0.0;
    if (mode == 3) {
        DeviceGuard guard(cx->device);
        FSI_TRY(measure_fp64_rate(cx->num_sms, cx->stream, &fp64_gflops));
    }
    if (mode == 1) {
        for (int k = 0; k < 8; ++k) {
            cx->prof_ms[k] = 0;
            cx->prof_n[k] = 0;
            cx->prof_work[k] = 0;
            cx->prof_gs64_bytes = 0;
        }
        cx->launch_base = launches_so_far();
        cx->profile = true;
    } else if (mode == 0) {
        cx->profile = false;
    }
    // algorithmic bytes of one fine-level smoother apply and residual SpMV
    const Problem &pb = cx->probs[0];
    const LevelDev &F = pb.dev.back();
    const double ts = cx->precision != FSI_FP64 ? 4.0 : 8.0;
    const double blk = smoother_bytes(*cx, F);
    const double spmv = spmv_bytes(F.A, ts);
    out[0] = (double)cx->prof_n[0];
    out[1] = cx->prof_ms[0];
    out[2] = blk;
    out[3] = (double)cx->prof_n[1];
    out[4] = cx->prof_ms[1];
    out[5] = spmv;
    out[6] = (double)(launches_so_far() - cx->launch_base);
    out[7] = (double)cx->prof_n[2];
    out[8] = cx->prof_ms[2];
    out[9] = (double)F.A.nnz * 12.0 + (double)(F.n + 1) * 4.0 + (double)F.n * 2.0 * 8.0;   // float64 A z
    out[10] = (double)F.A.nnz;
    out[11] = (double)cx->prof_n[3];
    out[12] = cx->prof_ms[3];
    double gj = 0.0;                                   // Gauss-Jordan inversion: 2 n^3 flops per block
    for (int64_t j = 0; j + 1 < (int64_t)F.h_blk_ptr.size(); ++j) {
        const double nj = (double)(F.h_blk_ptr[j + 1] - F.h_blk_ptr[j]);
        gj += 2.0 * nj * nj * nj;
    }
    out[13] = gj;
    out[14] = (double)F.n_blocks;
    // fine-level transfers (float32 cycle: 4-byte values and vectors)
    const LevelDev &Cl = pb.dev[pb.dev.size() >= 2 ? pb.dev.size() - 2 : 0];
    out[15] = (double)cx->prof_n[4];
    out[16] = cx->prof_ms[4];
    out[17] = (double)F.R.nnz * (ts + 4.0) + (double)(Cl.n + 1) * 4.0 + (double)F.n * ts + (double)Cl.n * ts;
    out[18] = (double)cx->prof_n[5];
    out[19] = cx->prof_ms[5];
    out[20] = (double)F.P.nnz * (ts + 4.0) + (double)(F.n + 1) * 4.0 + (double)Cl.n * ts + 2.0 * (double)F.n * ts;
    out[21] = fp64_gflops;
    out[22] = (double)cx->prof_n[6];
    out[23] = cx->prof_ms[6];
    out[24] = cx->prof_work[6];
    out[25] = (double)cx->prof_n[7];
    out[26] = cx->prof_ms[7];
    out[27] = cx->prof_work[7];
    out[28] = cx->prof_gs64_bytes;
    for (int k = 29; k < 32; ++k) out[k] = 0.0;
    return FSI_OK;
}

}  // extern "C"

namespace fsi {
namespace {
// Rebuild every binned-ELL copy of the context (level operators, transfers,
// their transposes and the cascade's operators, when present) with
// cx.ell_lanes lanes per row; captured graphs hold the old copies' pointers
// and are dropped.
fsi_status rebuild_ells(Context &cx) {
    cudaStream_t s = cx.stream;
    const bool conc = cx.probs.size() > 1;
    auto one = [&](DevCSR &A) -> fsi_status {
        if (A.nnz == 0 || !A.val64.p) return FSI_OK;
        FSI_TRY(build_ell(A, s, conc, cx.ell_lanes));
        A.ell.val32.release();
        if (A.val32.p) FSI_TRY(ell_fill_f32(A, s));
        return FSI_OK;
    };
    for (auto &pb : cx.probs) {
        drop_graphs(pb);
        for (auto &L : pb.dev) {
            for (DevCSR *A : {&L.A, &L.AT, &L.P, &L.R, &L.PT, &L.RT, &L.Ac, &L.ATc, &L.Rc, &L.RTc}) FSI_TRY(one(*A));
        }
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}
}  // namespace
}  // namespace fsi

extern "C" {

fsi_status fsi_autotune_layout(fsi_ctx *ctx, const int *lanes, int n_lanes, const fsi_solve_opts *opts, int *chosen,
                               double *times_ms) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !lanes || n_lanes < 1 || n_lanes > 8 || !chosen) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (!cx->smoothers_ready) { set_error("fsi_setup_smoothers has not completed"); return FSI_ERR_STATE; }
    FSI_TRY(check_opts(opts));
    for (int c = 0; c < n_lanes; ++c)
        if (!(lanes[c] == 0 || lanes[c] == 1 || lanes[c] == 4 || lanes[c] == 8 || lanes[c] == 16)) {
            set_error("lanes per row must be 0 (size rule), 1, 4, 8 or 16");
            return FSI_ERR_ARG;
        }
    DeviceGuard guard(cx->device);
    cudaStream_t s = cx->stream;
    const int np = (int)cx->probs.size();
    // right-hand sides b = A * 1 per problem (set-up time memory)
    std::vector<DevBuf> bv(np), xv(np);
    for (int i = 0; i < np; ++i) {
        Problem &pb = cx->probs[i];
        const int64_t n = pb.dev.back().n;
        DevBuf ones;
        FSI_TRY(ones.alloc((size_t)n * 8));
        FSI_TRY(bv[i].alloc((size_t)n * 8));
        FSI_TRY(xv[i].alloc((size_t)n * 8));
        std::vector<double> h1(n, 1.0);
        FSI_CUDA(cudaMemcpyAsync(ones.p, h1.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        const DevCSR &A = pb.dev.back().A;
        FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), ones.as<double>(), (const double *)nullptr,
                                                    bv[i].as<double>(), SPMV_SET, s));
        FSI_CUDA(cudaStreamSynchronize(s));
    }
    double best_t = 1e300;
    int best = lanes[0];
    for (int c = 0; c < n_lanes; ++c) {
        cx->ell_lanes = lanes[c];
        FSI_TRY(rebuild_ells(*cx));
        double t_ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {           // the first run captures the graphs
            std::vector<Run> runs(np);
            for (int i = 0; i < np; ++i) {
                runs[i].pb = &cx->probs[i];
                runs[i].b = bv[i].as<double>();
                runs[i].x = xv[i].as<double>();
                runs[i].o = *opts;
                runs[i].o.use_x0 = 0;
            }
            const auto t0 = std::chrono::steady_clock::now();
            fsi_status e = solve_runs(*cx, runs);
            FSI_CUDA(cudaStreamSynchronize(s));
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (e == FSI_ERR_CUDA || e == FSI_ERR_ALLOC) return e;
            t_ms = e == FSI_OK ? ms : 1e300;
        }
        if (times_ms) times_ms[c] = t_ms;
        if (t_ms < best_t) {
            best_t = t_ms;
            best = lanes[c];
        }
    }
    cx->ell_lanes = best;
    FSI_TRY(rebuild_ells(*cx));
    *chosen = best;
    g_last_error.clear();
    return FSI_OK;
}

fsi_status fsi_get_cost(fsi_ctx *ctx, int prob, double *cost) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !cost || prob < 0 || prob >= (int)cx->probs.size()) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (!cx->smoothers_ready) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    const Problem &pb = cx->probs[prob];
    const LevelDev &F = pb.dev.back();
    cost[0] = cycle_bytes(*cx, pb);
    cost[1] = (double)F.A.nnz * 12.0 + (double)(F.n + 1) * 4.0 + (double)F.n * 2.0 * 8.0;   // float64 A z
    cost[2] = (double)F.n * (cx->precision != FSI_FP64 ? 20.0 : 24.0);   // Gram-Schmidt, per basis vector
    cost[3] = (double)F.n;
    return FSI_OK;
}

fsi_status fsi_autotune(fsi_ctx *ctx, const int *candidates, int n_cand, const fsi_solve_opts *opts,
                        int *chosen, double *times_ms) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !candidates || n_cand < 1 || n_cand > 8 || !chosen) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (!cx->smoothers_ready) { set_error("fsi_setup_smoothers has not completed"); return FSI_ERR_STATE; }
    FSI_TRY(check_opts(opts));
    for (int c = 0; c < n_cand; ++c)
        if (candidates[c] < 1 || candidates[c] > 16) { set_error("candidate patch out of range"); return FSI_ERR_ARG; }
    DeviceGuard guard(cx->device);
    cudaStream_t s = cx->stream;
    const int np = (int)cx->probs.size();
    std::vector<int> done(np, 0);
    for (int i = 0; i < np; ++i) {
        if (done[i]) continue;
        // size class: same dimension, fine size and level count
        std::vector<int> cls;
        for (int k = i; k < np; ++k) {
            const ProblemDesc &a = cx->probs[i].desc, &b = cx->probs[k].desc;
            if (!done[k] && a.dim == b.dim && a.n_fine == b.n_fine && a.n_levels == b.n_levels) cls.push_back(k);
        }
        Problem &rep = cx->probs[i];
        const int64_t n = rep.dev.back().n;
        // right-hand side b = A * 1 and solution buffer (set-up time memory)
        DevBuf ones, bvec, xvec;
        FSI_TRY(ones.alloc((size_t)n * 8));
        FSI_TRY(bvec.alloc((size_t)n * 8));
        FSI_TRY(xvec.alloc((size_t)n * 8));
        std::vector<double> h1(n, 1.0);
        FSI_CUDA(cudaMemcpyAsync(ones.p, h1.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        const DevCSR &A = rep.dev.back().A;
        FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), ones.as<double>(), (const double *)nullptr,
                                                    bvec.as<double>(), SPMV_SET, s));
        FSI_CUDA(cudaStreamSynchronize(s));
        double best_t = 1e300;
        int best = candidates[0];
        for (int c = 0; c < n_cand; ++c) {
            rep.patch = candidates[c];
            FSI_TRY(setup_smoothers_problem(*cx, rep));
            double t_ms = 1e300;
            for (int rep_i = 0; rep_i < 2; ++rep_i) {     // first run captures the step graphs
                fsi_solve_stats st;
                fsi_status e = solve_one(*cx, rep, bvec.as<double>(), xvec.as<double>(), opts, &st, false);
                if (e == FSI_ERR_CUDA || e == FSI_ERR_ALLOC) return e;
                t_ms = (e == FSI_OK && st.converged) ? st.solve_ms : 1e300;
            }
            if (times_ms) times_ms[(size_t)i * n_cand + c] = t_ms;
            if (t_ms < best_t) {
                best_t = t_ms;
                best = candidates[c];
            }
        }
        for (int k : cls) {
            Problem &pb = cx->probs[k];
            pb.patch = best;
            FSI_TRY(setup_smoothers_problem(*cx, pb));
            chosen[k] = best;
            done[k] = 1;
            if (times_ms && k != i)
                for (int c = 0; c < n_cand; ++c) times_ms[(size_t)k * n_cand + c] = times_ms[(size_t)i * n_cand + c];
        }
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    g_last_error.clear();      // candidates that did not converge are not an error of the call
    return FSI_OK;
}

fsi_status fsi_get_sizes(const fsi_ctx *ctx, int prob, int level, int64_t *out) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || !out) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const LevelDev &D = pb->dev[level];
    const LevelHost &H = pb->host[level];
    out[0] = H.n_dofs;
    out[1] = D.A.nnz;
    out[2] = D.n_blocks;
    out[3] = D.max_block;
    for (int g = 0; g < 7; ++g) out[4 + g] = H.off[g];
    return FSI_OK;
}

fsi_status fsi_get_dof_map(const fsi_ctx *ctx, int prob, int level, int32_t *field, int32_t *comp, int32_t *node) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || !field || !comp || !node) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const LevelHost &H = pb->host[level];
    std::memcpy(field, H.dof_field.data(), H.n_dofs * 4);
    std::memcpy(comp, H.dof_comp.data(), H.n_dofs * 4);
    std::memcpy(node, H.dof_node.data(), H.n_dofs * 4);
    return FSI_OK;
}

fsi_status fsi_get_matrix(const fsi_ctx *ctx, int prob, int level, int64_t *row_ptr, int32_t *col, double *val) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || !row_ptr || !col || !val) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const Context *cx = reinterpret_cast<const Context *>(ctx);
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    HostCSR H;
    FSI_TRY(download_csr(pb->dev[level].A, H, cx->stream));
    std::memcpy(row_ptr, H.ptr.data(), H.ptr.size() * 8);
    std::memcpy(col, H.col.data(), H.col.size() * 4);
    std::memcpy(val, H.val.data(), H.val.size() * 8);
    return FSI_OK;
}

fsi_status fsi_get_transfer(const fsi_ctx *ctx, int prob, int level, int which, int64_t *row_ptr, int32_t *col,
                            double *val) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || level < 1 || !row_ptr || (which != 0 && which != 1)) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const HostCSR &H = which == 0 ? pb->hP[level] : pb->hR[level];
    std::memcpy(row_ptr, H.ptr.data(), H.ptr.size() * 8);
    if (col) std::memcpy(col, H.col.data(), H.col.size() * 4);
    if (val) std::memcpy(val, H.val.data(), H.val.size() * 8);
    return FSI_OK;
}

fsi_status fsi_get_blocks(const fsi_ctx *ctx, int prob, int level, int64_t *blk_ptr, int32_t *idx) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || level < 1 || !blk_ptr) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const LevelDev &D = pb->dev[level];
    if (D.h_blk_ptr.empty()) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    std::memcpy(blk_ptr, D.h_blk_ptr.data(), D.h_blk_ptr.size() * 8);
    if (idx) std::memcpy(idx, D.h_blk_idx.data(), D.h_blk_idx.size() * 4);
    return FSI_OK;
}

fsi_status fsi_get_block_passes(const fsi_ctx *ctx, int prob, int level, int32_t *pass) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || level < 1 || !pass) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    const LevelDev &D = pb->dev[level];
    if (D.h_blk_ptr.empty()) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    if (D.h_pass.size() + 1 != D.h_blk_ptr.size()) { set_error("monolithic (AS) blocks have no sweep passes"); return FSI_ERR_STATE; }
    std::memcpy(pass, D.h_pass.data(), D.h_pass.size() * 4);
    return FSI_OK;
}

fsi_status fsi_apply_operator(fsi_ctx *ctx, int prob, int level, const double *x, double *y) {
    Problem *pb = get_prob(ctx, prob, level);
    if (!pb || !x || !y) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    const DevCSR &A = pb->dev[level].A;
    FSI_TRY(launch_spmv<double, double, double>(A, A.val64.as<double>(), x, (const double *)nullptr, y, SPMV_SET,
                                                cx->stream));
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    return FSI_OK;
}

}  // extern "C"

// Working vectors of fsi_apply_smoother_noalloc: a file-scope device array
// (2 x FSI_NOALLOC_MAX_DOFS float64), shared by every call in the process.
static __device__ __align__(256) double g_noalloc_scratch[2 * (size_t)FSI_NOALLOC_MAX_DOFS];

namespace fsi {
namespace {
// device address of g_noalloc_scratch on the current device.  Looked up on
// every call (the host-side symbol is not a device address): the lookup
// allocates nothing, and a per-process cache would go stale if the device's
// primary context were reset and recreated.
fsi_status noalloc_scratch(double **out) {
    void *p = nullptr;
    FSI_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<double *>(p);
    return FSI_OK;
}

template <class T>
fsi_status apply_smoother_noalloc_t(Context &cx, LevelDev &L, const double *r, double *y, int tr, double *scratch) {
    cudaStream_t s = cx.stream;
    T *rt = reinterpret_cast<T *>(scratch);
    T *yt = reinterpret_cast<T *>(scratch + FSI_NOALLOC_MAX_DOFS);
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f64_f32(r, reinterpret_cast<float *>(rt), L.n, s));
    else FSI_CUDA(cudaMemcpyAsync(rt, r, (size_t)L.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaMemsetAsync(yt, 0, (size_t)L.n * sizeof(T), s));   // the array keeps the last call's data
    const double om = cx.omega;
    cx.omega = 1.0;   // plain P2^{-1} r
    fsi_status st = smooth_apply<T>(cx, L, rt, yt, tr != 0);
    cx.omega = om;
    FSI_TRY(st);
    if (std::is_same<T, float>::value) FSI_TRY(launch_cast_f32_f64(reinterpret_cast<const float *>(yt), y, L.n, s));
    else FSI_CUDA(cudaMemcpyAsync(y, yt, (size_t)L.n * 8, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}
}  // namespace
}  // namespace fsi

extern "C" {

fsi_status fsi_apply_smoother_noalloc(fsi_ctx *ctx, int prob, int level, const double *r, double *y, int transpose) {
    g_last_error.clear();
    Problem *pb = get_prob(ctx, prob, level);
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!pb || level < 1 || !r || !y) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (!cx->smoothers_ready) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    LevelDev &L = pb->dev[level];
    if (L.n > FSI_NOALLOC_MAX_DOFS) {
        set_error("level has " + std::to_string(L.n) + " dofs; fsi_apply_smoother_noalloc supports at most " +
                  std::to_string((long long)FSI_NOALLOC_MAX_DOFS));
        return FSI_ERR_ARG;
    }
    DeviceGuard guard(cx->device);
    double *scratch = nullptr;
    FSI_TRY(noalloc_scratch(&scratch));
    return cx->precision != FSI_FP64 ? apply_smoother_noalloc_t<float>(*cx, L, r, y, transpose, scratch)
                                      : apply_smoother_noalloc_t<double>(*cx, L, r, y, transpose, scratch);
}

fsi_status fsi_apply_smoother(fsi_ctx *ctx, int prob, int level, const double *r, double *y, int transpose) {
    Problem *pb = get_prob(ctx, prob, level);
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!pb || level < 1 || !r || !y) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (!cx->smoothers_ready) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    LevelDev &L = pb->dev[level];
    if (transpose && L.mult) FSI_TRY(build_transposes(*cx, *pb));
    return cx->precision != FSI_FP64 ? apply_smoother_t<float>(*cx, L, r, y, transpose)
                                      : apply_smoother_t<double>(*cx, L, r, y, transpose);
}

fsi_status fsi_apply_vcycle(fsi_ctx *ctx, int prob, const double *v, double *z, int transpose) {
    Problem *pb = get_prob(ctx, prob, 0);
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!pb || !v || !z) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (!cx->smoothers_ready) { set_error("smoothers not set up"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx->device);
    if (transpose) FSI_TRY(build_transposes(*cx, *pb));
    return cx->precision != FSI_FP64 ? apply_vcycle_t<float>(*cx, *pb, v, z, transpose)
                                      : apply_vcycle_t<double>(*cx, *pb, v, z, transpose);
}

void fsi_destroy(fsi_ctx *ctx) {
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx) return;
    if (cx->host_only) {
        delete cx;
        return;
    }
    {
        DeviceGuard guard(cx->device);
        cudaStreamSynchronize(cx->stream);
        if (cx->h_pinned) cudaFreeHost(cx->h_pinned);
        cx->h_pinned = nullptr;
        collect_marks(*cx);
        for (cudaEvent_t e : cx->ev_pool) cudaEventDestroy(e);
        cx->ev_pool.clear();
        for (int d = 0; d < 2; ++d) {
            if (cx->batch_graph[d]) cudaGraphExecDestroy(cx->batch_graph[d]);
            cx->batch_graph[d] = nullptr;
        }
        if (cx->cublas) cublasDestroy(static_cast<cublasHandle_t>(cx->cublas));
        cx->cublas = nullptr;
        for (auto &pb : cx->probs) {
            drop_graphs(pb);
            if (pb.stream) {
                cudaStreamSynchronize(pb.stream);
                cudaStreamDestroy(pb.stream);
                pb.stream = nullptr;
            }
            if (pb.h_scal) cudaFreeHost(pb.h_scal);
            pb.h_scal = nullptr;
            if (pb.h_fg) cudaFreeHost(pb.h_fg);
            pb.h_fg = nullptr;
            if (pb.ev_a) cudaEventDestroy(pb.ev_a);
            if (pb.ev_b) cudaEventDestroy(pb.ev_b);
            pb.ev_a = pb.ev_b = nullptr;
        }
        if (cx->work) cudaStreamSynchronize(cx->work);
        cx->probs.clear();
        cx->flags.release();
        if (cx->ev_in) cudaEventDestroy(cx->ev_in);
        if (cx->ev_out) cudaEventDestroy(cx->ev_out);
        if (cx->work) cudaStreamDestroy(cx->work);
        for (auto &c : cx->cap)
            if (c) cudaStreamDestroy(c);
    }
    delete cx;
}

}  // extern "C"

// ------------------------------------------------------------------ nonlinear
// Sec. 2.2: the residual of the nonlinear monolithic formulation and exact
// Newton on one time step.  Host code orders the launches (residual, norms,
// Jacobians on every level, block set-up, FGMRES, update) and reads one
// norm per Newton step; all arithmetic runs in the kernels.
namespace fsi {
namespace {

// level-lc dof -> level-(lc+1) dof at the coinciding node (-1: none there)
std::vector<int32_t> nl_injection(const LevelHost &F, const LevelHost &Cc) {
    std::vector<int32_t> map((size_t)Cc.n_dofs, -1);
    const int64_t mc2 = 2 * (int64_t)Cc.n + 1, mf2 = 2 * (int64_t)F.n + 1;
    for (int64_t y = 0; y < Cc.nq2; ++y) {
        const int64_t yf = (2 * (y / mc2)) * mf2 + 2 * (y % mc2);
        for (int i = 0; i < 2; ++i) {
            map[Cc.d_dof[y * 2 + i]] = F.d_dof[yf * 2 + i];
            map[Cc.v_dof[y * 2 + i]] = F.v_dof[yf * 2 + i];
        }
    }
    const int64_t mc1 = Cc.n + 1, mf1 = F.n + 1;
    for (int64_t z = 0; z < Cc.nq1; ++z) {
        const int64_t zf = (2 * (z / mc1)) * mf1 + 2 * (z % mc1);
        if (Cc.ps_dof[z] >= 0) map[Cc.ps_dof[z]] = F.ps_dof[zf];
        if (Cc.pf_dof[z] >= 0) map[Cc.pf_dof[z]] = F.pf_dof[zf];
    }
    return map;
}

fsi_status nl_setup_problem(Context &cx, Problem &pb, const fsi_nl_params &in) {
    cudaStream_t s = cx.stream;
    const ProblemDesc &d = pb.desc;
    NlParams &P = pb.nl;
    P.rho_s = d.rho_s;
    P.rho_f = d.rho_f;
    P.mu_f = d.mu_f;
    P.dt = d.dt;
    P.C1 = in.C1 > 0 ? in.C1 : d.mu_s / 3.0;
    P.C2 = in.C1 > 0 ? in.C2 : P.C1 / 2.0;
    P.k_ale = (double)d.n_fine * (double)d.n_fine;
    P.force = in.force;
    P.period = in.period;
    const int L = (int)pb.host.size();
    pb.nlev.clear();
    pb.nlev.resize(L);
    for (int l = 0; l < L; ++l) {
        const LevelHost &H = pb.host[l];
        NlLevelDev &N = pb.nlev[l];
        N.n = H.n;
        N.ds_end = (int32_t)H.off[1];
        FSI_TRY(upload(N.elem_dofs, H.elem_dofs.data(), H.elem_dofs.size() * 4, s));
        FSI_TRY(upload(N.material, H.material.data(), H.material.size(), s));
        FSI_TRY(upload(N.w, H.w.data(), H.w.size() * 8, s));
        // colours by the parity of the element coordinates; solid elements
        // first inside a colour (warps of one material)
        std::vector<int32_t> el;
        el.reserve((size_t)H.n_el);
        N.colour_ptr[0] = 0;
        for (int c = 0; c < 4; ++c) {
            for (int solid = 1; solid >= 0; --solid)
                for (int64_t e = 0; e < H.n_el; ++e) {
                    const int64_t ex = e % H.n, ey = e / H.n;
                    if ((int)((ex & 1) + 2 * (ey & 1)) == c && (H.material[e] != 0) == (solid == 1))
                        el.push_back((int32_t)e);
                }
            N.colour_ptr[c + 1] = (int64_t)el.size();
        }
        FSI_TRY(upload(N.elems, el.data(), el.size() * 4, s));
        size_t pbytes = 0;
        FSI_TRY(nl_point_bytes(N, &pbytes));
        FSI_TRY(N.pts.alloc(pbytes));
        FSI_TRY(launch_nl_positions(N, pb.dev[l].A, pb.dev[l].fixed.as<uint8_t>(), s));
        if (l + 1 < L) {
            const std::vector<int32_t> map = nl_injection(pb.host[l + 1], H);
            FSI_TRY(upload(N.inj, map.data(), map.size() * 4, s));
            FSI_TRY(N.U.alloc((size_t)H.n_dofs * 8));
            FSI_TRY(N.Un.alloc((size_t)H.n_dofs * 8));
        }
    }
    const int64_t n = pb.dev.back().n;
    FSI_TRY(pb.nl_R.alloc((size_t)n * 8));
    FSI_TRY(pb.nl_dU.alloc((size_t)n * 8));
    for (auto &f : pb.nl_fj) FSI_CUDA(f.create());
    FSI_TRY(pb.nl_coarse_work.alloc((size_t)pb.n0 * 2 * pb.n0 * 8));
    FSI_CUDA(cudaStreamSynchronize(s));
    pb.nl_ready = true;
    return FSI_OK;
}

// Jacobians of every level at U (level L-1) and the injected states, then
// the derived data of the operators: ELL values, coarse inverse; float32
// copies, transposes and the cascade's operators are rebuilt on demand.
fsi_status nl_assemble(Context &cx, Problem &pb, const double *U, const double *Un, double t_new) {
    cudaStream_t s = cx.stream;
    const int L = (int)pb.dev.size();
    std::vector<const double *> Us(L), Uns(L);
    Us[L - 1] = U;
    Uns[L - 1] = Un;
    for (int l = L - 2; l >= 0; --l) {
        NlLevelDev &N = pb.nlev[l];
        const uint8_t *fx = pb.dev[l].fixed.as<uint8_t>();
        FSI_TRY(launch_nl_inject(N.inj.as<int32_t>(), fx, Us[l + 1], N.U.as<double>(), pb.dev[l].n, s));
        FSI_TRY(launch_nl_inject(N.inj.as<int32_t>(), fx, Uns[l + 1], N.Un.as<double>(), pb.dev[l].n, s));
        Us[l] = N.U.as<double>();
        Uns[l] = N.Un.as<double>();
    }
    FSI_CUDA(cudaMemsetAsync(cx.flags.p, 0, 16, s));
    for (int l = 0; l < L; ++l) {
        LevelDev &D = pb.dev[l];
        FSI_TRY(launch_nl_jacobian(pb.nlev[l], pb.nl, D.fixed.as<uint8_t>(), D.A, Us[l], Uns[l], t_new,
                                   cx.flags.as<int>() + 3, s, pb.nl_fj));
        if (D.A.val32.p)                       // float32 copy in place (its address is in captured graphs)
            FSI_TRY(launch_cast_f64_f32(D.A.val64.as<double>(), D.A.val32.as<float>(), D.A.nnz, s));
        FSI_TRY(ell_refill(D.A, s));
    }
    int fw[4] = {0, 0, 0, 0};
    FSI_CUDA(cudaMemcpyAsync(fw, cx.flags.p, sizeof(fw), cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    if (fw[3]) {
        set_error("nonlinear Jacobian has an entry outside the operator pattern");
        return FSI_ERR_STATE;
    }
    FSI_CUDA(cudaMemsetAsync(cx.flags.p, 0, 16, s));
    FSI_TRY(coarse_invert(pb.dev[0].A, pb.n0, pb.coarse_inv.as<double>(), cx.flags.as<int>(), s,
                          pb.nl_coarse_work.as<double>()));
    int flag = 0;
    FSI_TRY(read_flag(cx, &flag));
    if (flag) {
        set_error("coarse-level Jacobian is singular");
        return FSI_ERR_ZERO_PIVOT;
    }
    pb.coarse_inv_t.release();
    pb.coarse_inv_c.release();
    pb.coarse_inv_ct.release();
    pb.transposes_ready = false;
    pb.cascade_ready = false;
    pb.dA_mu.release();
    pb.ops_changed = true;
    cx.smoothers_ready = false;
    return FSI_OK;
}

// The operators of one Newton step: the Jacobians of every level with the
// coarse inverse, then the in-place refactorisation of the Schwarz blocks.
// (Running the coarse levels' refactorisation beside the fine Jacobian on a
// second stream was measured: no gain on 256^2, the fine Jacobian's CTAs
// fill every SM.)
fsi_status nl_operators(Context &cx, Problem &pb, const double *U, const double *Un, double t_new, double *jac_ms,
                        double *setup_ms) {
    auto t0 = std::chrono::steady_clock::now();
    FSI_TRY(nl_assemble(cx, pb, U, Un, t_new));
    *jac_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    t0 = std::chrono::steady_clock::now();
    fsi_status e = refactor_smoothers(cx, pb);
    if (e == FSI_OK) FSI_CUDA(cudaStreamSynchronize(cx.stream));
    *setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return e;
}

// ||v||_2 on the host
fsi_status nl_norm(Context &cx, Problem &pb, const double *v, int64_t n, double *out) {
    FSI_TRY(norm2_to_host(cx, pb, v, n, 9));
    FSI_CUDA(cudaStreamSynchronize(cx.stream));
    *out = std::sqrt(pb.h_scal[9]);
    return FSI_OK;
}

Problem *nl_problem(fsi_ctx *ctx, int prob) {
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || cx->host_only || prob < 0 || prob >= (int)cx->probs.size()) return nullptr;
    return &cx->probs[prob];
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_nl_setup(fsi_ctx *ctx, const fsi_nl_params *params) {
    g_last_error.clear();
    Context *cx = reinterpret_cast<Context *>(ctx);
    if (!cx || !params) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (cx->host_only) { set_error("host-only context"); return FSI_ERR_STATE; }
    if (!cx->nonlinear) {
        set_error("the hierarchy was built without nonlinear patterns (fsi_hier_opts.nonlinear = 1)");
        return FSI_ERR_STATE;
    }
    if (!(params->period > 0) || !std::isfinite(params->force) || params->C2 < 0) {
        set_error("nonlinear parameters out of range");
        return FSI_ERR_ARG;
    }
    for (auto &pb : cx->probs)
        if (pb.desc.dim != 2) { set_error("the nonlinear residual is 2D"); return FSI_ERR_ARG; }
    DeviceGuard guard(cx->device);
    FSI_TRY(nl_upload_tables(cx->stream));
    for (auto &pb : cx->probs) FSI_TRY(nl_setup_problem(*cx, pb, *params));
    return FSI_OK;
}

fsi_status fsi_nl_residual(fsi_ctx *ctx, int prob, int level, const double *U, const double *Un, double t_new,
                           double *R) {
    g_last_error.clear();
    Problem *pb = nl_problem(ctx, prob);
    if (!pb || !U || !Un || !R || level < 0 || level >= (int)pb->dev.size() || R == U || R == Un) {
        set_error("invalid arguments");
        return FSI_ERR_ARG;
    }
    if (!pb->nl_ready) { set_error("fsi_nl_setup has not run"); return FSI_ERR_STATE; }
    Context *cx = reinterpret_cast<Context *>(ctx);
    DeviceGuard guard(cx->device);
    LevelDev &D = pb->dev[level];
    FSI_TRY(launch_nl_residual(pb->nlev[level], pb->nl, D.fixed.as<uint8_t>(), D.n, U, Un, t_new, R, cx->stream));
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    return FSI_OK;
}

fsi_status fsi_nl_inject(fsi_ctx *ctx, int prob, int level, const double *U_fine, double *U_coarse) {
    g_last_error.clear();
    Problem *pb = nl_problem(ctx, prob);
    if (!pb || !U_fine || !U_coarse || level < 1 || level >= (int)pb->dev.size()) {
        set_error("invalid arguments");
        return FSI_ERR_ARG;
    }
    if (!pb->nl_ready) { set_error("fsi_nl_setup has not run"); return FSI_ERR_STATE; }
    Context *cx = reinterpret_cast<Context *>(ctx);
    DeviceGuard guard(cx->device);
    FSI_TRY(launch_nl_inject(pb->nlev[level - 1].inj.as<int32_t>(), pb->dev[level - 1].fixed.as<uint8_t>(), U_fine,
                             U_coarse, pb->dev[level - 1].n, cx->stream));
    FSI_CUDA(cudaStreamSynchronize(cx->stream));
    return FSI_OK;
}

fsi_status fsi_nl_jacobian(fsi_ctx *ctx, int prob, const double *U, const double *Un, double t_new) {
    g_last_error.clear();
    Problem *pb = nl_problem(ctx, prob);
    if (!pb || !U || !Un) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (!pb->nl_ready) { set_error("fsi_nl_setup has not run"); return FSI_ERR_STATE; }
    Context *cx = reinterpret_cast<Context *>(ctx);
    DeviceGuard guard(cx->device);
    return nl_assemble(*cx, *pb, U, Un, t_new);
}

fsi_status fsi_nl_step(fsi_ctx *ctx, int prob, const double *Un, double *U, double t_new, const fsi_nl_opts *o,
                       fsi_nl_stats *st) {
    g_last_error.clear();
    const auto t_call = std::chrono::steady_clock::now();
    Problem *pbp = nl_problem(ctx, prob);
    if (!pbp || !Un || !U || !o || U == Un) { set_error("invalid arguments"); return FSI_ERR_ARG; }
    if (!(o->nl_rtol >= 0) || o->max_newton < 1 || o->max_newton > FSI_NL_MAX_NEWTON || !(o->lin_rtol > 0) ||
        o->restart < 1 || o->restart > 64 || o->max_iters < 1) {
        set_error("Newton options out of range");
        return FSI_ERR_ARG;
    }
    Problem &pb = *pbp;
    Context &cx = *reinterpret_cast<Context *>(ctx);
    if (!pb.nl_ready) { set_error("fsi_nl_setup has not run"); return FSI_ERR_STATE; }
    if (!cx.smoothers_configured) { set_error("fsi_setup_smoothers has not run"); return FSI_ERR_STATE; }
    DeviceGuard guard(cx.device);
    fsi_nl_stats S;
    std::memset(&S, 0, sizeof(S));
    cudaStream_t s = cx.stream;
    LevelDev &F = pb.dev.back();
    const int64_t n = F.n;
    FSI_TRY(ensure_workspace(cx, pb, o->restart));
    double *R = pb.nl_R.as<double>(), *dU = pb.nl_dU.as<double>();
    FSI_TRY(launch_nl_residual(pb.nlev.back(), pb.nl, F.fixed.as<uint8_t>(), n, U, Un, t_new, R, s));
    double res = 0.0;
    FSI_TRY(nl_norm(cx, pb, R, n, &res));
    const double r0 = res;
    S.residual[0] = res;
    fsi_status status = FSI_ERR_NOT_CONVERGED;
    fsi_solve_opts lo{};
    lo.rtol = o->lin_rtol;
    lo.restart = o->restart;
    lo.max_iters = o->max_iters;
    lo.use_x0 = 0;
    for (int k = 0;; ++k) {
        if (!std::isfinite(res)) { status = FSI_ERR_NONFINITE; set_error("non-finite nonlinear residual"); break; }
        if (res <= o->nl_rtol * std::max(r0, 1e-300) || res == 0.0) { status = FSI_OK; S.converged = 1; break; }
        if (k == o->max_newton) break;
        fsi_status e = nl_operators(cx, pb, U, Un, t_new, &S.jacobian_ms, &S.setup_ms);
        if (e != FSI_OK) { status = e; break; }
        cx.smoothers_ready = std::none_of(cx.probs.begin(), cx.probs.end(),
                                          [](const Problem &q) { return q.ops_changed; });
        FSI_TRY(launch_nl_axpby(R, R, -1.0, 0.0, n, s));      // R <- -R
        const auto t0 = std::chrono::steady_clock::now();
        fsi_solve_stats ls{};
        e = solve_one(cx, pb, R, dU, &lo, &ls, false);
        S.solve_ms += ms_since(t0);
        S.lin_iterations[k] = ls.iterations;
        S.lin_rho[k] = ls.rho;
        S.newton_steps = k + 1;
        if (e != FSI_OK) { status = e; break; }
        FSI_TRY(launch_nl_axpby(U, dU, 1.0, 1.0, n, s));      // U <- U + dU
        FSI_TRY(launch_nl_residual(pb.nlev.back(), pb.nl, F.fixed.as<uint8_t>(), n, U, Un, t_new, R, s));
        FSI_TRY(nl_norm(cx, pb, R, n, &res));
        S.residual[k + 1] = res;
    }
    FSI_CUDA(cudaStreamSynchronize(s));
    S.status = status;
    S.total_ms = ms_since(t_call);
    if (st) *st = S;
    if (status == FSI_ERR_NOT_CONVERGED && g_last_error.empty())
        set_error("Newton did not reach the nonlinear tolerance in max_newton steps");
    return status;
}

}  // extern "C"
