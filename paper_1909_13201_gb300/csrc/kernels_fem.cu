// Element assembly of the level operators (Sec. 2.2 weak form, linearised)
// and small elementwise kernels.
//
// One CTA per element.  The frozen advection w and its gradient are first
// evaluated at the 4^dim Gauss points into shared memory; then every
// (row, column) pair of the element's local dofs that the weak form couples
// is integrated by the Gauss rule and added into the CSR value array
// (float64 atomics; the row's columns are sorted, the position is found by
// binary search).  Coupling rules by local row kind (J2 rows, Eq. matrix_J2):
//   solid element: S row d(a,i) <- d (2 mu_s eps:eps), u comp i (rho_s/dt mass), p^s (-div);
//                  K row u(a,i) <- u(a,i) (lumped mass), d(a,i) (-lumped mass/dt);
//                  V row p(al)  <- d (-div), p^s (-(1/lambda_s) mass)
//   fluid element: momentum row (S at solid-class, F at fluid-class nodes)
//                  <- u (rho_f/dt mass + rho_f advection + mu_f (grad+grad^T)), p^f (-div),
//                     d (-(rho_f/dt) (d.grad) w);
//                  A row d(a,i) at fluid-class nodes <- d (k (grad+grad^T), k = 1/V_el fine);
//                  W row p(al) <- u (-div)
// Fixed rows and columns are skipped; fixed rows get a unit diagonal after.
#include "context.h"

namespace fsi {

namespace {

struct AsmParams {
    int dim, n2, n1, nq, nloc;
    int64_t nq2;
    double h, mu_s, lambda_s, rho_s, rho_f, mu_f, dt, k_ale;
    int mu_derivative;
    int32_t ds_end;          // dofs below this index are d^s (solid-class d)
    const int32_t *elem_dofs;
    const uint8_t *material;
    const uint8_t *fixed;
    const double *w;         // dim x nq2 nodal advection of the level
    const int32_t *elem_q2;  // n_el x n2 Q2 node indices (for w lookup)
    const double *wq, *phi, *dphi, *psi;
    const int32_t *row_ptr, *col;
    double *val;
    int *err;
};

__device__ __forceinline__ int find_col(const int32_t *col, int lo, int hi, int c) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// kind of local dof: 0 d, 1 u, 2 p ; local node a and component i
__device__ __forceinline__ void local_kind(int loc, int n2, int dim, int &kind, int &a, int &i) {
    if (loc < n2 * dim) { kind = 0; a = loc / dim; i = loc % dim; }
    else if (loc < 2 * n2 * dim) { kind = 1; a = (loc - n2 * dim) / dim; i = (loc - n2 * dim) % dim; }
    else { kind = 2; a = loc - 2 * n2 * dim; i = 0; }
}

__global__ void assemble_kernel(AsmParams P) {
    extern __shared__ double sm[];
    const int e = blockIdx.x;
    const int dim = P.dim, n2 = P.n2, n1 = P.n1, nq = P.nq, nloc = P.nloc;
    double *wqv = sm;                    // [k][q]   w_k at q
    double *gw = sm + dim * nq;          // [i][j][q] reference d_j w_i at q
    const int32_t *ed = P.elem_dofs + (size_t)e * nloc;
    const bool solid = P.material[e] != 0;
    const int32_t *nodes = P.elem_q2 + (size_t)e * n2;
    if (!solid && !P.mu_derivative) {
        for (int t = threadIdx.x; t < dim * nq; t += blockDim.x) {
            const int k = t / nq, q = t % nq;
            double s = 0.0;
            for (int c = 0; c < n2; ++c) s += P.w[(size_t)k * P.nq2 + nodes[c]] * P.phi[q * n2 + c];
            wqv[t] = s;
        }
        for (int t = threadIdx.x; t < dim * dim * nq; t += blockDim.x) {
            const int i = t / (dim * nq), j = (t / nq) % dim, q = t % nq;
            double s = 0.0;
            for (int c = 0; c < n2; ++c)
                s += P.w[(size_t)i * P.nq2 + nodes[c]] * P.dphi[(q * dim + j) * n2 + c];
            gw[t] = s;
        }
    }
    __syncthreads();
    const double h = P.h;
    double J = 1.0;
    for (int k = 0; k < dim; ++k) J *= h;        // element volume h^dim
    const double Jg = J / h, Jgg = J / (h * h);
    for (int pr = threadIdx.x; pr < nloc * nloc; pr += blockDim.x) {
        const int rl = pr / nloc, cl = pr % nloc;
        const int32_t R = ed[rl], C = ed[cl];
        if (R < 0 || C < 0) continue;
        if (P.fixed[R] || P.fixed[C]) continue;
        int rk, a, i, ck, b, j;
        local_kind(rl, n2, dim, rk, a, i);
        local_kind(cl, n2, dim, ck, b, j);
        const bool node_solid = (rk < 2) && (ed[a * dim] < P.ds_end);   // d dof of node a in d^s
        double v = 0.0;
        bool hit = false;
        if (P.mu_derivative) {
            if (!(solid && rk == 0 && ck == 0)) continue;
            hit = true;
            for (int q = 0; q < nq; ++q) {
                double lap = 0.0;
                for (int k = 0; k < dim; ++k) lap += P.dphi[(q * dim + k) * n2 + a] * P.dphi[(q * dim + k) * n2 + b];
                const double t = (i == j ? lap : 0.0) + P.dphi[(q * dim + j) * n2 + a] * P.dphi[(q * dim + i) * n2 + b];
                v += P.wq[q] * t;
            }
            v *= Jgg;
        } else if (solid) {
            if (rk == 0) {                                   // S row
                if (ck == 0) {
                    hit = true;
                    for (int q = 0; q < nq; ++q) {
                        double lap = 0.0;
                        for (int k = 0; k < dim; ++k) lap += P.dphi[(q * dim + k) * n2 + a] * P.dphi[(q * dim + k) * n2 + b];
                        const double t = (i == j ? lap : 0.0) + P.dphi[(q * dim + j) * n2 + a] * P.dphi[(q * dim + i) * n2 + b];
                        v += P.wq[q] * t;
                    }
                    v *= P.mu_s * Jgg;
                } else if (ck == 1) {
                    if (i != j) continue;
                    hit = true;
                    for (int q = 0; q < nq; ++q) v += P.wq[q] * P.phi[q * n2 + a] * P.phi[q * n2 + b];
                    v *= P.rho_s / P.dt * J;
                } else {
                    hit = true;
                    for (int q = 0; q < nq; ++q) v += P.wq[q] * P.psi[q * n1 + b] * P.dphi[(q * dim + i) * n2 + a];
                    v *= -Jg;
                }
            } else if (rk == 1) {                            // K row: lumped, diagonal
                if (a != b || i != j || ck == 2) continue;
                hit = true;
                double lump = 0.0;
                for (int q = 0; q < nq; ++q) lump += P.wq[q] * P.phi[q * n2 + a];
                lump *= J;
                v = (ck == 1) ? lump : -lump / P.dt;
            } else {                                         // V row
                if (ck == 0) {
                    hit = true;
                    for (int q = 0; q < nq; ++q) v += P.wq[q] * P.psi[q * n1 + a] * P.dphi[(q * dim + j) * n2 + b];
                    v *= -Jg;
                } else if (ck == 2) {
                    hit = true;
                    for (int q = 0; q < nq; ++q) v += P.wq[q] * P.psi[q * n1 + a] * P.psi[q * n1 + b];
                    v *= -J / P.lambda_s;
                } else continue;
            }
        } else {
            const int nqv = nq;
            const double *wqp = wqv;
            const double *gwp = gw;
            const bool momentum = (rk == 0 && node_solid) || (rk == 1 && !node_solid);
            if (momentum) {
                if (ck == 1) {
                    hit = true;
                    double mass = 0.0, adv = 0.0, visc = 0.0;
                    for (int q = 0; q < nqv; ++q) {
                        const double pa = P.phi[q * n2 + a], pb = P.phi[q * n2 + b];
                        double wg = 0.0, lap = 0.0;
                        for (int k = 0; k < dim; ++k) {
                            wg += wqp[k * nqv + q] * P.dphi[(q * dim + k) * n2 + b];
                            lap += P.dphi[(q * dim + k) * n2 + a] * P.dphi[(q * dim + k) * n2 + b];
                        }
                        mass += P.wq[q] * pa * pb;
                        adv += P.wq[q] * pa * wg;
                        visc += P.wq[q] * ((i == j ? lap : 0.0) + P.dphi[(q * dim + j) * n2 + a] * P.dphi[(q * dim + i) * n2 + b]);
                    }
                    v = P.mu_f * Jgg * visc;
                    if (i == j) v += P.rho_f / P.dt * J * mass + P.rho_f * Jg * adv;
                } else if (ck == 2) {
                    hit = true;
                    for (int q = 0; q < nqv; ++q) v += P.wq[q] * P.psi[q * n1 + b] * P.dphi[(q * dim + i) * n2 + a];
                    v *= -Jg;
                } else {
                    hit = true;
                    for (int q = 0; q < nqv; ++q)
                        v += P.wq[q] * P.phi[q * n2 + a] * P.phi[q * n2 + b] * gwp[(i * dim + j) * nqv + q];
                    v *= -(P.rho_f / P.dt) * Jg;
                }
            } else if (rk == 0) {                            // A row (fluid-class node)
                if (ck != 0) continue;
                hit = true;
                for (int q = 0; q < nqv; ++q) {
                    double lap = 0.0;
                    for (int k = 0; k < dim; ++k) lap += P.dphi[(q * dim + k) * n2 + a] * P.dphi[(q * dim + k) * n2 + b];
                    const double t = (i == j ? lap : 0.0) + P.dphi[(q * dim + j) * n2 + a] * P.dphi[(q * dim + i) * n2 + b];
                    v += P.wq[q] * t;
                }
                v *= P.k_ale * Jgg;
            } else if (rk == 2) {                            // W row
                if (ck != 1) continue;
                hit = true;
                for (int q = 0; q < nqv; ++q) v += P.wq[q] * P.psi[q * n1 + a] * P.dphi[(q * dim + j) * n2 + b];
                v *= -Jg;
            } else continue;                                  // K row gets nothing from fluid
        }
        if (!hit) continue;
        const int pos = find_col(P.col, P.row_ptr[R], P.row_ptr[R + 1], C);
        if (pos < 0) { atomicExch(P.err, 1); continue; }
        atomicAdd(&P.val[pos], v);
    }
}

__global__ void cast_f64_f32_kernel(const double *__restrict__ s, float *__restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}
__global__ void cast_f32_f64_kernel(const float *__restrict__ s, double *__restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

__global__ void set_fixed_diag_kernel(const int32_t *ptr, const int32_t *col, const uint8_t *fixed,
                                      double *val, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (!fixed[r]) continue;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) val[k] = (col[k] == r) ? 1.0 : 0.0;
    }
}

__global__ void pattern_grad_kernel(const int32_t *ptr, const int32_t *col, const double *lam,
                                    const double *x, double *out, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double l = lam[r];
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) out[k] = -l * x[col[k]];
    }
}

// 1/A_ii for the Jacobi rows (u^s and fixed dofs), stored in float64 and float32
__global__ void jacobi_setup_kernel(const int32_t *ptr, const int32_t *col, const double *val,
                                    const int32_t *idx, int64_t n, double *d64, float *d32) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int r = idx[k];
        double d = 0.0;
        for (int q = ptr[r]; q < ptr[r + 1]; ++q)
            if (col[q] == r) d = val[q];
        const double inv = 1.0 / d;
        if (d64) d64[k] = inv;
        if (d32) d32[k] = (float)inv;
    }
}

inline int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

fsi_status launch_assemble(const LevelHost &L, const ProblemDesc &p, const RefTables &ref,
                           const DevCSR &A, bool mu_derivative, double *val_out, cudaStream_t s) {
    const int dim = L.dim;
    const int n2 = ref.n2, n1 = ref.n1, nq = ref.nq;
    // element -> Q2 nodes (for w)
    std::vector<int32_t> eq2((size_t)L.n_el * n2);
    for (int64_t e = 0; e < L.n_el; ++e) {
        int64_t c[3], r = e;
        for (int k = 0; k < dim; ++k) { c[k] = r % L.n; r /= L.n; }
        const int64_t m2 = 2 * (int64_t)L.n + 1;
        for (int a = 0; a < n2; ++a) {
            int64_t ai[3] = {a % 3, (a / 3) % 3, (a / 9) % 3};
            int64_t idx = 0;
            for (int k = dim - 1; k >= 0; --k) idx = idx * m2 + 2 * c[k] + ai[k];
            eq2[(size_t)e * n2 + a] = (int32_t)idx;
        }
    }
    DevBuf d_ed, d_mat, d_fixed, d_w, d_eq2, d_wq, d_phi, d_dphi, d_psi, d_err;
    FSI_TRY(d_ed.alloc(L.elem_dofs.size() * 4));
    FSI_TRY(d_mat.alloc(L.material.size()));
    FSI_TRY(d_fixed.alloc(L.fixed.size()));
    FSI_TRY(d_w.alloc(L.w.size() * 8));
    FSI_TRY(d_eq2.alloc(eq2.size() * 4));
    FSI_TRY(d_wq.alloc(ref.wq.size() * 8));
    FSI_TRY(d_phi.alloc(ref.phi.size() * 8));
    FSI_TRY(d_dphi.alloc(ref.dphi.size() * 8));
    FSI_TRY(d_psi.alloc(ref.psi.size() * 8));
    FSI_TRY(d_err.alloc(4));
    FSI_CUDA(cudaMemcpyAsync(d_ed.p, L.elem_dofs.data(), L.elem_dofs.size() * 4, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_mat.p, L.material.data(), L.material.size(), cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_fixed.p, L.fixed.data(), L.fixed.size(), cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_w.p, L.w.data(), L.w.size() * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_eq2.p, eq2.data(), eq2.size() * 4, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_wq.p, ref.wq.data(), ref.wq.size() * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_phi.p, ref.phi.data(), ref.phi.size() * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_dphi.p, ref.dphi.data(), ref.dphi.size() * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(d_psi.p, ref.psi.data(), ref.psi.size() * 8, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemsetAsync(d_err.p, 0, 4, s));
    FSI_CUDA(cudaMemsetAsync(val_out, 0, (size_t)A.nnz * 8, s));
    AsmParams P;
    P.dim = dim; P.n2 = n2; P.n1 = n1; P.nq = nq; P.nloc = L.nloc; P.nq2 = L.nq2;
    P.h = L.h; P.mu_s = p.mu_s; P.lambda_s = p.lambda_s; P.rho_s = p.rho_s; P.rho_f = p.rho_f;
    P.mu_f = p.mu_f; P.dt = p.dt;
    P.k_ale = 1.0;
    for (int k = 0; k < dim; ++k) P.k_ale *= (double)p.n_fine;   // 1/V_el of the fine element
    P.mu_derivative = mu_derivative ? 1 : 0;
    P.ds_end = (int32_t)L.off[1];
    P.elem_dofs = d_ed.as<int32_t>(); P.material = d_mat.as<uint8_t>(); P.fixed = d_fixed.as<uint8_t>();
    P.w = d_w.as<double>(); P.elem_q2 = d_eq2.as<int32_t>();
    P.wq = d_wq.as<double>(); P.phi = d_phi.as<double>(); P.dphi = d_dphi.as<double>(); P.psi = d_psi.as<double>();
    P.row_ptr = A.ptr.as<int32_t>(); P.col = A.col.as<int32_t>(); P.val = val_out; P.err = d_err.as<int>();
    const size_t smem = (size_t)(dim * nq + dim * dim * nq) * 8;
    assemble_kernel<<<(unsigned)L.n_el, 256, smem, s>>>(P);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    if (!mu_derivative) {
        set_fixed_diag_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                                      d_fixed.as<uint8_t>(), val_out, A.n_rows);
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    int herr = 0;
    FSI_CUDA(cudaMemcpyAsync(&herr, d_err.p, 4, cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("assembly produced an entry outside the operator pattern");
        return FSI_ERR_STATE;
    }
    return FSI_OK;
}

fsi_status launch_cast_f64_f32(const double *src, float *dst, int64_t n, cudaStream_t s) {
    cast_f64_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
fsi_status launch_cast_f32_f64(const float *src, double *dst, int64_t n, cudaStream_t s) {
    cast_f32_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
fsi_status launch_set_fixed_diag(const DevCSR &A, const uint8_t *fixed, double *val, cudaStream_t s) {
    set_fixed_diag_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                                  fixed, val, A.n_rows);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}
fsi_status launch_jacobi_setup(const DevCSR &A, const int32_t *idx, int64_t n, double *d64, float *d32,
                               cudaStream_t s) {
    if (n == 0) return FSI_OK;
    jacobi_setup_kernel<<<grid_for(n, 256), 256, 0, s>>>(A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                         A.val64.as<double>(), idx, n, d64, d32);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_pattern_grad(const DevCSR &A, const double *lam, const double *x, double *out,
                               cudaStream_t s) {
    pattern_grad_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.ptr.as<int32_t>(), A.col.as<int32_t>(),
                                                                lam, x, out, A.n_rows);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

}  // namespace fsi
