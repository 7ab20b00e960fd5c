// Device-side data of a solver context and the internal kernel interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fsi.h"
#include "host_setup.h"

namespace fsi {

// Last-error message (thread local) and CUDA checks that turn into statuses.
void set_error(const std::string &msg);
#define FSI_CUDA(...)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (__VA_ARGS__);                                                \
        if (e_ != cudaSuccess) {                                                       \
            ::fsi::set_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
            return FSI_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)
#define FSI_TRY(...)                       \
    do {                                   \
        fsi_status s_ = (__VA_ARGS__);     \
        if (s_ != FSI_OK) return s_;       \
    } while (0)

// An auxiliary stream with a fork and a join event (owned): the two field
// systems of a multiplicative sweep run side by side on it and the caller's
// stream.  Inside a stream capture the fork/join become graph edges.
struct ForkJoin {
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ForkJoin() = default;
    ForkJoin(const ForkJoin &) = delete;
    ForkJoin &operator=(const ForkJoin &) = delete;
    ForkJoin(ForkJoin &&o) noexcept { *this = std::move(o); }
    ForkJoin &operator=(ForkJoin &&o) noexcept {
        if (this != &o) {
            release();
            aux = o.aux; fork = o.fork; join = o.join;
            o.aux = nullptr; o.fork = nullptr; o.join = nullptr;
        }
        return *this;
    }
    ~ForkJoin() { release(); }
    void release() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (aux) cudaStreamDestroy(aux);
        aux = nullptr; fork = nullptr; join = nullptr;
    }
    cudaError_t create() {
        if (aux) return cudaSuccess;
        cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        return e;
    }
};

// Owned device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    fsi_status alloc(size_t nbytes) {
        release();
        if (nbytes == 0) nbytes = 16;
        if (cudaMalloc(&p, nbytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of " + std::to_string(nbytes) + " bytes failed");
            p = nullptr;
            return FSI_ERR_ALLOC;
        }
        bytes = nbytes;
        return FSI_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Length-binned ELL copy of a CSR operator, the layout the solve-path
// products stream.  Rows are sorted by their number of nonzeros (stable, so
// rows of one length keep their order) and grouped into bins of equal
// length; bin b stores its rows column-major, entry k of sorted row t at
// off + k * stride + t with stride = rows rounded up to a slab of 32 / G
// rows (G lanes per row), so with G = 1 a warp of 32 consecutive rows reads
// every entry position as one coalesced 128-byte line and needs no row
// pointers.  Padding entries hold column 0, value 0.
struct EllBin {
    int64_t off;          // first stored entry of the bin
    int32_t rows, len;    // rows in the bin, nonzeros per row
    int32_t stride;       // rows rounded up to a multiple of 32 / G
    int32_t first;        // position of the bin's first row in perm
    int32_t slab0;        // first slab (32 / G rows) of the bin
    int32_t pad;
};
struct DevEll {
    int nbins = 0;
    int G = 1;                      // lanes per row (slab = 32 / G rows)
    bool stream = true;             // evict-first loads (operators far larger than L2 share)
    int64_t nslabs = 0, size = 0;   // slabs (warps), stored entries (with padding)
    int64_t nnz = 0;                // entries of the operator (without padding)
    DevBuf bins;                    // EllBin[nbins]
    DevBuf perm;                    // int32[n_rows]: CSR row of each sorted position
    DevBuf col;                     // int32[size]
    DevBuf val64, val32;            // copies of the CSR val64 / val32
    DevBuf fbase, fstride;          // fill map: first ELL position (int64) and stride (int32) of every CSR row
};

// CSR on the device: int32 row pointers and columns, float64 values and
// (mixed precision) a float32 copy; `ell` holds the binned-ELL copy used by
// the SpMV whenever the values passed are val64 or val32.
struct DevCSR {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    DevBuf ptr, col, val64, val32;
    int group = 8;        // threads per row in the CSR SpMV kernel
    DevEll ell;
};

// One pass of the locally multiplicative sweep: apply work items [it0, it1)
// of its level, field 0 (displacement, solid pressure) or 1 (velocity, fluid
// pressure), the rows its blocks (or Jacobi rows) cover, and the binned-ELL
// copies of A_FF (and A_FF^T) restricted to those rows.
struct SweepPass {
    int64_t it0 = 0, it1 = 0;
    int field = 0;
    bool jacobi = false;
    std::vector<int32_t> rows;
    DevEll ell, ell_t;
};

struct LevelDev {
    int64_t n = 0;
    DevCSR A, AT;         // operator and (adjoint) its transpose
    DevCSR P, R;          // l >= 1: P_l (n_l x n_{l-1}), R_l (n_{l-1} x n_l)
    DevCSR PT, RT;        // adjoint: P^T (restriction), R^T (prolongation)
    // swapped cascade (Sec. 5): the same-system diagonal blocks of A and R
    // (entries coupling the displacement and velocity systems removed) and
    // their transposes; P couples no systems and is used as it is
    DevCSR Ac, ATc, Rc, RTc;
    DevBuf fixed;         // uint8 per dof
    // Schwarz blocks (l >= 1)
    int64_t n_blocks = 0, max_block = 0, inv_elems = 0;
    std::vector<int64_t> h_blk_ptr;
    std::vector<int32_t> h_blk_idx;
    std::vector<int32_t> h_pass;                // field split: sweep pass of every block (block order)
    DevBuf blk_ptr, blk_idx, blk_off, blk_w;   // int32, int32, int64, working-precision weights
    DevBuf inv;                                 // block inverses, row-major, padded rows
    DevBuf inv_scale;                           // float16 storage: float32 scale per block row
    int inv_store = 0;                          // 0 float64, 1 float32, 2 float16 + row scale
    int64_t n_items = 0;
    DevBuf items;                               // int4 (block, row begin, row end, 0) apply work items
    // owner-computes combination of overlapping blocks (additive levels):
    // stage has one slot per entry of blk_idx; owner d = own_dof[d] sums its
    // slots own_pos[own_ptr[d] .. own_ptr[d+1]) (block order) times own_w[d]
    int64_t n_own = 0;
    DevBuf stage, own_dof, own_ptr, own_pos, own_w;
    int64_t n_jac = 0;
    DevBuf jac_idx, jac_inv;                    // int32, working precision 1/diag
    // V-cycle vectors in working precision
    DevBuf b, x, r;
    // locally multiplicative sweep (mult != 0): blocks sorted by pass, one
    // pass per (kind, colour) plus the Jacobi rows, in sweep order
    int mult = 0;
    bool mult_t_ready = false;
    std::vector<SweepPass> passes;
    DevBuf y, rr;                               // correction (zero between sweeps), pass residual
    ForkJoin fj;                                // the velocity system's passes run on fj.aux
    std::vector<uint8_t> h_keep[2];             // per dof: free dof of field 0 (d, p^s) / 1 (u, p^f)
    DevBuf keep[2];
};

// Control block of a device-driven FGMRES solve (one per problem, device
// memory).  The host writes rtol/max_iters/m before a launch and reads the
// rest afterwards; the kernels of the solve graph update it in between.
struct FgState {
    int k = 0;              // Arnoldi columns completed in the current cycle
    int its = 0;            // total Arnoldi steps
    int cycles = 0;         // completed restart cycles
    int flags = 0;          // bit 0: non-finite value met
    int max_iters = 0, m = 0;
    int pad0 = 0, pad1 = 0;
    double rtol = 0.0;
    double bnorm = 0.0, beta = 0.0, r0 = 0.0;
};

// Nonlinear problem (Sec. 2.2): physical data of the residual
struct NlParams {
    double rho_s = 1, rho_f = 1, mu_f = 1, dt = 1;
    double C1 = 0, C2 = 0;      // Mooney-Rivlin constants
    double k_ale = 1;           // harmonic-extension coefficient (1/V_el of the fine element)
    double force = 0, period = 1;   // body force F0 sin(2 pi t / period) w(x)
};

// Per level of the nonlinear problem: element tables, elements by colour
// (parity of the element coordinates; solid elements first inside a
// colour), the injection map from the next finer level and the injected
// states of the coarse levels.
struct NlLevelDev {
    int n = 0;
    int32_t ds_end = 0;             // first d^f dof
    DevBuf elem_dofs;               // int32 n_el x 40
    DevBuf material;                // uint8 n_el
    DevBuf w;                       // float64 2 x nq2: spatial profile of the body force
    DevBuf elems;                   // int32 n_el, colour-major
    int64_t colour_ptr[5] = {0, 0, 0, 0, 0};
    DevBuf inj;                     // int32 n (l < L-1): dof of level l+1 at the coinciding node, -1 none
    DevBuf U, Un;                   // float64 states (l < L-1: injected)
    DevBuf pts;                     // point scratch of the Jacobian: n_el x 9 records
    DevBuf pos;                     // int32 n_el x 40 x 40: CSR position of each element-matrix entry
};

struct Problem {
    ProblemDesc desc;
    int patch = 1;                   // Vanka group edge of this problem's smoothers
    std::vector<LevelHost> host;
    std::vector<LevelDev> dev;       // index = level
    std::vector<HostCSR> hP, hR;     // host transfers (for accessors)
    int64_t n0 = 0;                  // coarse size
    DevBuf coarse_inv;               // n0 x n0 float64 inverse of A_0 (row-major)
    DevBuf coarse_inv_t;             // its transpose (transposed cycle; built with the transposes)
    DevBuf coarse_inv_c, coarse_inv_ct;   // swapped cascade: inverse of A_0's system blocks, transpose
    bool cascade_ready = false;      // Ac / Rc / coarse_inv_c built
    DevBuf coarse_b, coarse_x;       // float64 coarse vectors
    DevBuf dA_mu;                    // float64 values of dA/dmu_s on the fine pattern
    bool transposes_ready = false;
    // Krylov workspace (fine level)
    int m_alloc = 0;
    DevBuf V, Z, H, g, cs, sn, y, w, rvec, xwork, partials, scal, h1, h2;
    DevBuf V32;                      // float32 copy of the basis (first Gram-Schmidt pass, mixed modes)
    // one CUDA graph per Arnoldi step j (index 0: forward, 1: transposed)
    std::vector<cudaGraphExec_t> graphs[2];
    cudaStream_t stream = nullptr;   // the problem's own solve stream
    double *h_scal = nullptr;        // pinned scalars of the running solve
    std::vector<int64_t> graph_kernels[2];
    // device-driven solve: one graph per direction (nested WHILE nodes),
    // control block, fixed copies of b, x and z_j, per-solve timing events
    cudaGraphExec_t solve_graph[2] = {nullptr, nullptr};
    int solve_graph_m[2] = {0, 0};
    int64_t graph_counts[2][3] = {{0, 0, 0}, {0, 0, 0}};   // kernels: prologue, per cycle, per step
    DevBuf fg, bbuf, xbuf, zbuf;
    FgState *h_fg = nullptr;         // pinned: [0] parameters in, [1] state out
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // nonlinear problem (fsi_nl_setup)
    bool nl_ready = false;
    bool ops_changed = false;        // operators replaced since this problem's smoothers were set up
    std::vector<double> smoother_sig;   // options of the last full smoother set-up (empty: none)
    NlParams nl;
    std::vector<NlLevelDev> nlev;    // index = level
    DevBuf nl_R, nl_dU;              // fine residual (negated for the solve) and Newton update
    ForkJoin nl_fj[2];               // side streams of the Jacobian's seed kinds
    DevBuf nl_coarse_work;           // n0 x 2 n0 float64: the coarse inverse's working storage
};

// kernels launched by the library (all contexts), for launch accounting
void count_launch(int n = 1);
int64_t launches_so_far();

// Programmatic dependent launch (V-cycle kernels).  A kernel launched with
// launch_pdl may start while its predecessor on the stream is still
// running: it calls pdl_trigger() on entry (so that its own successor can
// be scheduled as soon as all of its CTAs run), does only work that reads
// no data of earlier kernels (static matrices, block inverses, work items),
// then pdl_wait(), which returns once every earlier kernel has completed
// and its writes are visible.  Nothing is written before pdl_wait().  Both
// are no-ops for a normal launch.  FSI_PDL=0 turns the attribute off.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
bool pdl_enabled();
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

struct Context {
    int device = 0;
    cudaStream_t stream = nullptr;
    int restriction = 0;
    int nonlinear = 0;               // patterns of the nonlinear residual's Jacobian
    int precision = FSI_FP64;
    int patch = 1;
    double omega = 1.0;
    int nu_pre = 1, nu_post = 1;
    int factor = FSI_FACTOR_AUTO;    // block inversion method (resolved per precision)
    int variant = FSI_SMOOTHER_FS;   // field-split (FS) or monolithic (AS) Schwarz blocks
    int mult_levels = 0;             // finest levels with the locally multiplicative sweep
    int cascade = 0;                 // 1: swapped cascade, the cycle on the two system blocks (Sec. 5)
    int ell_lanes = 0;               // lanes per row of every ELL copy (0: size rule; fsi_autotune_layout)
    void *cublas = nullptr;          // cuBLAS handle (batched GEMMs of the split inversion of large AS blocks)
    bool smoothers_ready = false;
    bool smoothers_configured = false;   // fsi_setup_smoothers completed once (its options are set)
    bool host_only = false;          // inspection context without device state
    std::vector<Problem> probs;
    DevBuf flags;                    // int32[4]: zero pivot, nonfinite, ...
    int num_sms = 152;
    int64_t *h_pinned = nullptr;     // pinned host scratch for scalars
    // profiling of fine-level launches (fsi_profile)
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;   // kind, start/stop
    // fine smoother, fine residual SpMV, outer float64 A z, fine block
    // inversion (set-up), fine restriction, fine prolongation, float64
    // Gram-Schmidt passes (work: FMAs), first Gram-Schmidt pass (work: bytes)
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double prof_work[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double prof_gs64_bytes = 0;      // bytes the float64 Gram-Schmidt passes must move (basis, w)
    int64_t launch_base = 0;
    // solves run on a context-owned non-blocking stream
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool use_graphs = true;
    bool device_loop = true;         // whole solve as one graph with WHILE nodes
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};   // streams for capturing loop bodies
    // batched solves: every problem's solve chain in one graph (per direction),
    // valid while no problem's graphs were dropped since (graph epoch)
    cudaGraphExec_t batch_graph[2] = {nullptr, nullptr};
    int batch_graph_m[2] = {0, 0};
    int64_t batch_epoch[2] = {-1, -1};
};

// ---------------------------------------------------------------- kernels
// (launch wrappers; all asynchronous on the given stream)
fsi_status launch_assemble(const LevelHost &L, const ProblemDesc &p, const RefTables &ref,
                           const DevCSR &A, bool mu_derivative, double *val_out, cudaStream_t s);
fsi_status launch_cast_f64_f32(const double *src, float *dst, int64_t n, cudaStream_t s);
fsi_status launch_cast_f32_f64(const float *src, double *dst, int64_t n, cudaStream_t s);

enum SpmvMode { SPMV_SET = 0, SPMV_RESID = 1, SPMV_ADD = 2 };
// y = A x | y = b - A x | y += A x ; matrix precision follows TA, vectors TX/TY
// zero_out (optional, length n_rows): set to 0 by the same launch (folds the
// zeroing of the next level's correction into the restriction)
template <class TA, class TX, class TY>
fsi_status launch_spmv(const DevCSR &A, const TA *val, const TX *x, const TY *b, TY *y, int mode,
                       cudaStream_t s, TY *zero_out = nullptr);
// v = 0 (normal launch; triggers its programmatic dependents at entry)
template <class T>
fsi_status launch_zero(T *v, int64_t n, cudaStream_t s);

// binned-ELL copy of A (structure and val64; val32 too if present), and
// the float32 copy of an existing ELL from A.val32.  concurrent: A belongs
// to one problem of a batch (its launches share the GPU with the others').
// force_G: lanes per row (1, 4, 8 or 16) chosen by the layout autotuner; 0 = the size rule
fsi_status build_ell(DevCSR &A, cudaStream_t s, bool concurrent, int force_G = 0);
fsi_status build_ell_subset(const DevCSR &A, const HostCSR &pat, const std::vector<int32_t> &rows,
                            const std::vector<uint8_t> &keep, const uint8_t *d_keep, DevEll &E,
                            cudaStream_t s, bool concurrent);
template <class T>
fsi_status launch_ell_resid(const DevEll &E, const T *x, const T *b, T *y, cudaStream_t s);
template <class T>
fsi_status launch_axpy_clear(T *x, T *y, T a, int64_t n, cudaStream_t s);
fsi_status ell_fill_f32(DevCSR &A, cudaStream_t s);

// storage: 0 float64, 1 float32, 2 float16 with a float32 scale per row
fsi_status launch_block_invert(const DevCSR &A, const LevelDev &lev, int storage, int *flags,
                               cudaStream_t s, int num_sms);
template <class T>
fsi_status launch_block_apply(const LevelDev &lev, const T *r, T *x, T omega, int transpose,
                              cudaStream_t s, int64_t it0 = 0, int64_t it1 = -1);
template <class T>
fsi_status launch_jacobi_apply(const LevelDev &lev, const T *r, T *x, T omega, cudaStream_t s);

// blocked float32 Gauss-Jordan (tensor: tcgen05 TF32 rank-32 updates;
// otherwise float32 FMAs); storage 1 float32, 2 float16 + row scale
// Monolithic blocks beyond one cluster (3D AS): inverse from the 2 x 2 split
// over the two field systems (off3 = first velocity-system dof), float32
fsi_status launch_block_invert_schur(Context &cx, const DevCSR &A, const LevelDev &lev, int64_t off3, bool tensor,
                                     int *flags, cudaStream_t s);
bool gj_tc_plan(int n, int *C_out, int *R_out, size_t *smem_out);
fsi_status launch_block_invert_tc(const DevCSR &A, const LevelDev &lev, int storage, bool tensor, int *flags,
                                  cudaStream_t s);

// work: n0 x 2 n0 float64 scratch (nullable: a temporary, and the call
// synchronises the stream before freeing it)
fsi_status coarse_invert(const DevCSR &A0, int64_t n0, double *inv, int *flags, cudaStream_t s,
                         double *work = nullptr);
// t = m^T for an n x n row-major float64 matrix
fsi_status launch_transpose(const double *m, int64_t n, double *t, cudaStream_t s);

template <class T>
fsi_status launch_dense_gemv(const double *M, int64_t n, const T *x, T *y, int transpose,
                             cudaStream_t s);

// Krylov helpers.  Where a control block `fg` is passed, the column index
// j (number of vectors nv = j + 1, count k) is read from fg->k on the device
// instead of the host argument, so one captured launch serves every step of
// a device-side loop; the host argument then only bounds the template size.
fsi_status launch_mdot(const double *V, int64_t ld, int nv, const double *w, int64_t n,
                       double *partials, int nblocks, cudaStream_t s, const FgState *fg = nullptr);
// V32 (optional, mixed modes): float32 copy of the basis for float32 dots in pass 2
fsi_status launch_update_dot(double *w, const double *V, int64_t ld, int nv, const double *h,
                             int64_t n, double *partials, int nblocks, int norm_only,
                             cudaStream_t s, const FgState *fg = nullptr, const float *V32 = nullptr);
fsi_status launch_reduce_partials(const double *partials, int nblocks, int nv, double *out,
                                  int accumulate, cudaStream_t s, const FgState *fg = nullptr);
fsi_status launch_givens(double *H, int ld, int j, const double *h1, const double *h2,
                         const double *hn2, double *cs, double *sn, double *g, double *scal,
                         cudaStream_t s, FgState *fg = nullptr, cudaGraphConditionalHandle loop = 0);
// v = w / scal[idx] (and its float32 copy v32 when non-null)
fsi_status launch_scale_copy(const double *w, double *v, const double *scal, int idx, int64_t n,
                             cudaStream_t s, const FgState *fg = nullptr, int64_t ld = 0, float *v32 = nullptr);
// float64 FMA throughput of the device (GFLOP/s, 2 flops per FMA)
fsi_status measure_fp64_rate(int num_sms, cudaStream_t s, double *gflops);
// first Gram-Schmidt pass from the float32 copy of the basis (mixed modes)
fsi_status launch_mdot32(const float *V, int64_t ld, int nv, const double *w, int64_t n, double *partials,
                         int nblocks, cudaStream_t s, const FgState *fg = nullptr);
fsi_status launch_backsolve(const double *H, int ld, int k, const double *g, double *y,
                            cudaStream_t s, const FgState *fg = nullptr);
template <class T>
fsi_status launch_combine(double *x, const T *Z, int64_t ld, int k, const double *y, int64_t n,
                          cudaStream_t s, const FgState *fg = nullptr);
fsi_status launch_init_basis(const double *r, double *v0, double *g, int m, const double *nrm2,
                             int64_t n, cudaStream_t s, FgState *fg = nullptr,
                             cudaGraphConditionalHandle loop = 0, float *v0f = nullptr);
// device-loop helpers: dst = (TO) V[:, fg->k]; zfix = Z[:, fg->k] = (double) z
// take_column also selects the Gram-Schmidt variant of the step (SWITCH
// node `sel`, value nv_class(fg->k + 1)) when sel is nonzero, and sets
// zero[0..n) = 0 when zero is non-null (the cycle's fine correction)
template <class TI, class TO>
fsi_status launch_take_column(const TI *V, int64_t ld, const FgState *fg, TO *dst, int64_t n, cudaStream_t s,
                              cudaGraphConditionalHandle sel = 0, TO *zero = nullptr);
// Gram-Schmidt kernels are instantiated for nv <= 1, 2, 4, 8, 16, 32, 65
constexpr int NV_CLASSES = 7;
__host__ __device__ inline int nv_class_bound(int c) { return c < 6 ? (1 << c) : 65; }
template <class T>
fsi_status launch_store_column(const T *z, double *zfix, double *Z, int64_t ld, const FgState *fg, int64_t n,
                               cudaStream_t s);
// loop control (one thread): after ||b||^2 (scal[5]) and ||r0||^2 (scal[6]);
// after the true residual of a cycle (scal[6])
fsi_status launch_fg_start(const double *scal, FgState *fg, cudaGraphConditionalHandle outer, cudaStream_t s);
fsi_status launch_fg_cycle(const double *scal, FgState *fg, cudaGraphConditionalHandle outer, cudaStream_t s);
fsi_status launch_pattern_grad(const DevCSR &A, const double *lam, const double *x, double *out,
                               cudaStream_t s);
fsi_status launch_jacobi_setup(const DevCSR &A, const int32_t *idx, int64_t n, double *d64, float *d32,
                               cudaStream_t s);
fsi_status launch_set_fixed_diag(const DevCSR &A, const uint8_t *fixed, double *val, cudaStream_t s);

// nonlinear residual and exact Jacobian (kernels_nl.cu)
fsi_status nl_upload_tables(cudaStream_t s);
fsi_status launch_nl_residual(const NlLevelDev &L, const NlParams &P, const uint8_t *fixed, int64_t n_dofs,
                              const double *U, const double *Un, double t_new, double *R, cudaStream_t s);
fsi_status launch_nl_jacobian(const NlLevelDev &L, const NlParams &P, const uint8_t *fixed, const DevCSR &A,
                              const double *U, const double *Un, double t_new, int *err, cudaStream_t s,
                              ForkJoin *fj);
// the element-matrix -> CSR position table of a level (built once; the pattern is fixed)
fsi_status launch_nl_positions(NlLevelDev &L, const DevCSR &A, const uint8_t *fixed, cudaStream_t s);
// bytes of a level's point scratch
fsi_status nl_point_bytes(const NlLevelDev &L, size_t *bytes);
fsi_status launch_nl_inject(const int32_t *map, const uint8_t *fixed_c, const double *Uf, double *Uc, int64_t nc,
                            cudaStream_t s);
// y = a x + b y (float64)
fsi_status launch_nl_axpby(double *y, const double *x, double a, double b, int64_t n, cudaStream_t s);
// re-fill the float64 (and, when present, float32) values of A's binned-ELL copy from its CSR values
fsi_status ell_refill(DevCSR &A, cudaStream_t s);
// the same for a row-subset copy built by build_ell_subset (same column mask)
fsi_status ell_subset_refill(const DevCSR &A, DevEll &E, const uint8_t *d_keep, cudaStream_t s);

}  // namespace fsi
