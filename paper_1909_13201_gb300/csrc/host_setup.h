// Host-side structure of the GMG hierarchy: levels, J2 numbering, sparsity
// patterns, transfer operators and Schwarz block index sets.  Integer and
// interpolation-weight work done once at set-up; all numerics of the solve
// (assembly values, factorisations, the V-cycle, FGMRES) run in CUDA kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fsi {

struct HostCSR {
    int64_t n_rows = 0, n_cols = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;     // empty for a pattern
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// One grid level (Sec. 3.3: midpoint refinement of a structured coarse grid).
struct LevelHost {
    int dim = 2, n = 0;          // n elements per direction
    double h = 0;
    int64_t n_el = 0, nq2 = 0, nq1 = 0;
    std::vector<uint8_t> material;          // n_el, 1 solid
    std::vector<uint8_t> q2_solid;          // solid-class Q2 node (touches a solid element)
    std::vector<uint8_t> q1_s, q1_f;        // vertex carries p^s / p^f
    std::vector<uint8_t> d_fixed, v_fixed;  // per Q2 node
    std::vector<int32_t> d_dof, v_dof;      // nq2 * dim
    std::vector<int32_t> ps_dof, pf_dof;    // nq1, -1 if absent
    int64_t off[7] = {0};                   // J2 group offsets d^s d^f p^s u^s u^f p^f
    int64_t n_dofs = 0;
    std::vector<uint8_t> fixed;             // n_dofs
    std::vector<int32_t> dof_field, dof_comp, dof_node;
    std::vector<double> w;                  // dim * nq2 advection (zero at solid-class nodes)
    std::vector<int32_t> elem_dofs;         // n_el * nloc local-to-global map (-1 none)
    int nloc = 0;                           // 2 * 3^dim * dim + 2^dim
    HostCSR pattern;                        // sparsity of A_l (fixed rows: diagonal only)
    bool nl_pattern = false;                // W rows also couple to d (Jacobian of the nonlinear residual)
    int64_t group_of(int64_t dof) const;
};

struct ProblemDesc {
    int dim, n_fine, n_levels, bc_preset;
    std::vector<uint8_t> material;
    std::vector<double> advection;          // dim * nq2_fine
    double mu_s, lambda_s, rho_s, rho_f, mu_f, dt;
    int nonlinear = 0;                      // patterns of the nonlinear residual's Jacobian (Sec. 2.2)
};

// Build levels 0 (coarse) .. L-1 (fine) with numbering, fixed sets,
// per-level advection, element dof tables and operator patterns.
std::string build_levels(const ProblemDesc &p, std::vector<LevelHost> &levels);

// P_l (fine x coarse) and the restriction R_l (coarse x fine).
void build_prolongation(const LevelHost &fine, const LevelHost &coarse, HostCSR &P);
void build_restriction(const HostCSR &P, const LevelHost &fine, const LevelHost &coarse,
                       bool classical, HostCSR &R);

// Schwarz block index sets of a level (Vanka groups of b^dim pressure
// vertices): field split (solid [d^s, p^s], fluid [d^f], fluid [u^f, p^f]
// per group) or, monolithic, one block of all fields per group (AS).
// tags (optional): per block its vertex group and kind (0 solid, 1 fluid-d,
// 2 fluid-u).
void build_blocks(const LevelHost &lev, int b, std::vector<int64_t> &blk_ptr,
                  std::vector<int32_t> &blk_idx, bool monolithic = false,
                  std::vector<int32_t> *tags = nullptr);

// Locally multiplicative sweep (Sec. 3.2): the pass of every field-split
// block, kind * k^dim + colour, where the colour of vertex group t is
// sum_a (t_a mod k) k^a and k = colour_period(b) is the smallest period that
// leaves two element layers between same-colour groups (4 for b = 1, 3 for
// b = 2, else 2).  Blocks of one pass share no entry of their field's
// operator, so a pass updates all its blocks at once and equals the paper's
// one-block-after-another update in that order.
int colour_period(int b);
void sweep_passes(const LevelHost &lev, int b, const std::vector<int32_t> &tags, std::vector<int32_t> &pass);

// Reference-cell tables of the 4-point Gauss rule: weights, Q2 values and
// gradients, Q1 values; layout [q][a], [q][k][a], [q][al].
struct RefTables {
    int dim, nq, n2, n1;
    std::vector<double> wq, phi, dphi, psi;
};
RefTables make_ref_tables(int dim);

}  // namespace fsi
