// Host-side structure of the hierarchy (see host_setup.h).
//
// Paper passages: Sec. 3.3 (levels by midpoint refinement, the same
// fluid/solid decomposition on every level -- a coarse element is solid when
// any descendant is), Eq. matrix_J2 (J2 ordering d^s d^f p^s u^s u^f p^f,
// interface test functions in the solid rows), Sec. 3.2 (Vanka block rule),
// Sec. 3.3 (P2 natural injection, R2 equation-aware restriction).
#include "host_setup.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

namespace fsi {

namespace {

inline int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// coordinates of flat index idx in an m^dim lattice (x fastest)
inline void unflat(int64_t idx, int64_t m, int dim, int64_t *c) {
    for (int k = 0; k < dim; ++k) {
        c[k] = idx % m;
        idx /= m;
    }
}
inline int64_t toflat(const int64_t *c, int64_t m, int dim) {
    int64_t r = 0;
    for (int k = dim - 1; k >= 0; --k) r = r * m + c[k];
    return r;
}

// Q2 Lagrange basis on [0,1], nodes 0, 1/2, 1
inline void q2_basis(double t, double v[3], double d[3]) {
    v[0] = 2.0 * (t - 0.5) * (t - 1.0);
    v[1] = 4.0 * t * (1.0 - t);
    v[2] = 2.0 * t * (t - 0.5);
    d[0] = 4.0 * t - 3.0;
    d[1] = 4.0 - 8.0 * t;
    d[2] = 4.0 * t - 1.0;
}

// elements of an n^dim grid whose closure contains the point with
// (half-)integer lattice coordinates pos in units of `unit` lattice steps per
// element (unit = 2 for Q2 nodes, 1 for Q1 vertices).  Returns the count.
int touching_elements(const int64_t *pos, int unit, int64_t n, int dim, int64_t *out) {
    int64_t lo[3], hi[3];
    for (int k = 0; k < dim; ++k) {
        // element i spans [unit*i, unit*(i+1)]
        int64_t a = (pos[k] - 1) / unit;  // candidate below when pos on a boundary
        if (pos[k] == 0) a = 0;
        int64_t b = pos[k] / unit;
        if (b > n - 1) b = n - 1;
        if (a < 0) a = 0;
        lo[k] = std::min(a, b);
        hi[k] = std::max(a, b);
    }
    int cnt = 0;
    int64_t c[3];
    for (int64_t z = lo[dim > 2 ? 2 : 0]; z <= (dim > 2 ? hi[2] : lo[0]); ++z) {
        (void)z;
        break;
    }
    // iterate the (at most 2^dim) candidate boxes
    int64_t span[3] = {1, 1, 1};
    for (int k = 0; k < dim; ++k) span[k] = hi[k] - lo[k] + 1;
    int64_t total = span[0] * span[1] * span[2];
    for (int64_t t = 0; t < total; ++t) {
        int64_t r = t;
        bool ok = true;
        for (int k = 0; k < dim; ++k) {
            c[k] = lo[k] + r % span[k];
            r /= span[k];
            if (!(unit * c[k] <= pos[k] && pos[k] <= unit * (c[k] + 1))) ok = false;
        }
        if (ok) out[cnt++] = toflat(c, n, dim);
    }
    return cnt;
}

}  // namespace

int64_t LevelHost::group_of(int64_t dof) const {
    int g = 0;
    while (g < 5 && dof >= off[g + 1]) ++g;
    return g;
}

RefTables make_ref_tables(int dim) {
    RefTables t;
    t.dim = dim;
    // 4-point Gauss-Legendre on [-1,1] mapped to [0,1] (exact to degree 7:
    // the advection integrand phi_a (d phi_b) phi_c has degree 6 per direction)
    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    const double x1[4] = {0.5 - 0.5 * b, 0.5 - 0.5 * a, 0.5 + 0.5 * a, 0.5 + 0.5 * b};
    const double w1[4] = {0.5 * wb, 0.5 * wa, 0.5 * wa, 0.5 * wb};
    t.nq = (int)ipow(4, dim);
    t.n2 = (int)ipow(3, dim);
    t.n1 = (int)ipow(2, dim);
    t.wq.assign(t.nq, 0.0);
    t.phi.assign((size_t)t.nq * t.n2, 0.0);
    t.dphi.assign((size_t)t.nq * dim * t.n2, 0.0);
    t.psi.assign((size_t)t.nq * t.n1, 0.0);
    for (int q = 0; q < t.nq; ++q) {
        int qi[3] = {q % 4, (q / 4) % 4, (q / 16) % 4};
        double v[3][3], d[3][3], l[3][2];
        double w = 1.0;
        for (int k = 0; k < dim; ++k) {
            q2_basis(x1[qi[k]], v[k], d[k]);
            l[k][0] = 1.0 - x1[qi[k]];
            l[k][1] = x1[qi[k]];
            w *= w1[qi[k]];
        }
        t.wq[q] = w;
        for (int aa = 0; aa < t.n2; ++aa) {
            int ai[3] = {aa % 3, (aa / 3) % 3, (aa / 9) % 3};
            double val = 1.0;
            for (int k = 0; k < dim; ++k) val *= v[k][ai[k]];
            t.phi[(size_t)q * t.n2 + aa] = val;
            for (int g = 0; g < dim; ++g) {
                double dv = 1.0;
                for (int k = 0; k < dim; ++k) dv *= (k == g) ? d[k][ai[k]] : v[k][ai[k]];
                t.dphi[((size_t)q * dim + g) * t.n2 + aa] = dv;
            }
        }
        for (int al = 0; al < t.n1; ++al) {
            double val = 1.0;
            for (int k = 0; k < dim; ++k) val *= l[k][(al >> k) & 1];
            t.psi[(size_t)q * t.n1 + al] = val;
        }
    }
    return t;
}

static void fill_level(LevelHost &L, const ProblemDesc &p) {
    const int dim = L.dim;
    const int64_t n = L.n, m2 = 2 * n + 1, m1 = n + 1;
    L.h = 1.0 / (double)n;
    L.n_el = ipow(n, dim);
    L.nq2 = ipow(m2, dim);
    L.nq1 = ipow(m1, dim);
    const int n2 = (int)ipow(3, dim), n1 = (int)ipow(2, dim);

    // node classes
    L.q2_solid.assign(L.nq2, 0);
    L.q1_s.assign(L.nq1, 0);
    L.q1_f.assign(L.nq1, 0);
    int64_t ec[3], c[3];
    for (int64_t e = 0; e < L.n_el; ++e) {
        unflat(e, n, dim, ec);
        const bool s = L.material[e] != 0;
        for (int aa = 0; aa < n2; ++aa) {
            int64_t ai[3] = {aa % 3, (aa / 3) % 3, (aa / 9) % 3};
            for (int k = 0; k < dim; ++k) c[k] = 2 * ec[k] + ai[k];
            if (s) L.q2_solid[toflat(c, m2, dim)] = 1;
        }
        for (int al = 0; al < n1; ++al) {
            for (int k = 0; k < dim; ++k) c[k] = ec[k] + ((al >> k) & 1);
            (s ? L.q1_s : L.q1_f)[toflat(c, m1, dim)] = 1;
        }
    }
    // boundary conditions
    L.d_fixed.assign(L.nq2, 0);
    L.v_fixed.assign(L.nq2, 0);
    for (int64_t y = 0; y < L.nq2; ++y) {
        unflat(y, m2, dim, c);
        bool lo[3] = {false, false, false}, hi[3] = {false, false, false};
        for (int k = 0; k < dim; ++k) {
            lo[k] = c[k] == 0;
            hi[k] = c[k] == m2 - 1;
        }
        if (p.bc_preset == 0) {
            const bool any = lo[0] || hi[0] || lo[1] || hi[1];
            if (L.q2_solid[y]) {
                L.d_fixed[y] = L.v_fixed[y] = (lo[0] || hi[0] || lo[1]);
            } else {
                L.d_fixed[y] = any;
                L.v_fixed[y] = lo[0] || lo[1] || hi[1];
            }
        } else {
            const bool f = lo[0] || lo[1] || hi[1] || lo[2] || hi[2];
            L.d_fixed[y] = L.v_fixed[y] = f;
        }
    }
    // J2 numbering
    int64_t ns = 0, nf = 0, nps = 0, npf = 0;
    for (int64_t y = 0; y < L.nq2; ++y) (L.q2_solid[y] ? ns : nf)++;
    for (int64_t z = 0; z < L.nq1; ++z) {
        nps += L.q1_s[z];
        npf += L.q1_f[z];
    }
    const int64_t sizes[6] = {ns * dim, nf * dim, nps, ns * dim, nf * dim, npf};
    L.off[0] = 0;
    for (int g = 0; g < 6; ++g) L.off[g + 1] = L.off[g] + sizes[g];
    L.n_dofs = L.off[6];
    L.d_dof.assign(L.nq2 * dim, -1);
    L.v_dof.assign(L.nq2 * dim, -1);
    L.ps_dof.assign(L.nq1, -1);
    L.pf_dof.assign(L.nq1, -1);
    int64_t cs = 0, cf = 0;
    for (int64_t y = 0; y < L.nq2; ++y) {
        for (int i = 0; i < dim; ++i) {
            if (L.q2_solid[y]) {
                L.d_dof[y * dim + i] = (int32_t)(L.off[0] + cs * dim + i);
                L.v_dof[y * dim + i] = (int32_t)(L.off[3] + cs * dim + i);
            } else {
                L.d_dof[y * dim + i] = (int32_t)(L.off[1] + cf * dim + i);
                L.v_dof[y * dim + i] = (int32_t)(L.off[4] + cf * dim + i);
            }
        }
        (L.q2_solid[y] ? cs : cf)++;
    }
    int64_t ks = 0, kf = 0;
    for (int64_t z = 0; z < L.nq1; ++z) {
        if (L.q1_s[z]) L.ps_dof[z] = (int32_t)(L.off[2] + ks++);
        if (L.q1_f[z]) L.pf_dof[z] = (int32_t)(L.off[5] + kf++);
    }
    L.fixed.assign(L.n_dofs, 0);
    L.dof_field.assign(L.n_dofs, 0);
    L.dof_comp.assign(L.n_dofs, 0);
    L.dof_node.assign(L.n_dofs, 0);
    for (int64_t y = 0; y < L.nq2; ++y)
        for (int i = 0; i < dim; ++i) {
            int32_t dd = L.d_dof[y * dim + i], vv = L.v_dof[y * dim + i];
            L.dof_field[dd] = 0; L.dof_comp[dd] = i; L.dof_node[dd] = (int32_t)y;
            L.dof_field[vv] = 1; L.dof_comp[vv] = i; L.dof_node[vv] = (int32_t)y;
            if (L.d_fixed[y]) L.fixed[dd] = 1;
            if (L.v_fixed[y]) L.fixed[vv] = 1;
        }
    for (int64_t z = 0; z < L.nq1; ++z) {
        if (L.ps_dof[z] >= 0) {
            L.dof_field[L.ps_dof[z]] = 2; L.dof_comp[L.ps_dof[z]] = 0; L.dof_node[L.ps_dof[z]] = (int32_t)z;
        }
        if (L.pf_dof[z] >= 0) {
            L.dof_field[L.pf_dof[z]] = 2; L.dof_comp[L.pf_dof[z]] = 1; L.dof_node[L.pf_dof[z]] = (int32_t)z;
        }
    }
    // advection sampled at the level's nodes from the fine nodes, zero in the solid
    const int64_t stride = p.n_fine / n, mf = 2 * (int64_t)p.n_fine + 1, nq2f = ipow(mf, dim);
    L.w.assign((size_t)dim * L.nq2, 0.0);
    for (int64_t y = 0; y < L.nq2; ++y) {
        if (L.q2_solid[y]) continue;
        unflat(y, m2, dim, c);
        int64_t cf3[3];
        for (int k = 0; k < dim; ++k) cf3[k] = c[k] * stride;
        const int64_t yf = toflat(cf3, mf, dim);
        for (int k = 0; k < dim; ++k) L.w[(size_t)k * L.nq2 + y] = p.advection[(size_t)k * nq2f + yf];
    }
    // element local dof tables: [d(a,i)] [v(a,i)] [p(al)] (p: the element's material copy)
    L.nloc = 2 * n2 * dim + n1;
    L.elem_dofs.assign((size_t)L.n_el * L.nloc, -1);
    for (int64_t e = 0; e < L.n_el; ++e) {
        unflat(e, n, dim, ec);
        int32_t *ed = &L.elem_dofs[(size_t)e * L.nloc];
        for (int aa = 0; aa < n2; ++aa) {
            int64_t ai[3] = {aa % 3, (aa / 3) % 3, (aa / 9) % 3};
            for (int k = 0; k < dim; ++k) c[k] = 2 * ec[k] + ai[k];
            const int64_t y = toflat(c, m2, dim);
            for (int i = 0; i < dim; ++i) {
                ed[aa * dim + i] = L.d_dof[y * dim + i];
                ed[n2 * dim + aa * dim + i] = L.v_dof[y * dim + i];
            }
        }
        for (int al = 0; al < n1; ++al) {
            for (int k = 0; k < dim; ++k) c[k] = ec[k] + ((al >> k) & 1);
            const int64_t z = toflat(c, m1, dim);
            ed[2 * n2 * dim + al] = L.material[e] ? L.ps_dof[z] : L.pf_dof[z];
        }
    }
}

// Column set of one row: the union over the elements touching the row's
// node of the columns the element couples to that row (same rule set as the
// assembly kernel), fixed columns dropped; fixed rows keep their diagonal.
static void build_pattern(LevelHost &L) {
    const int dim = L.dim;
    const int64_t n = L.n, m2 = 2 * n + 1, m1 = n + 1;
    const int n2 = (int)ipow(3, dim), n1 = (int)ipow(2, dim);
    const int nloc = L.nloc;
    std::vector<std::vector<int32_t>> rows(L.n_dofs);
#pragma omp parallel
    {
        std::vector<int32_t> cols;
        int64_t c[3], els[8];
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = 0; r < L.n_dofs; ++r) {
            cols.clear();
            if (L.fixed[r]) {
                rows[r].assign(1, (int32_t)r);
                continue;
            }
            const int f = L.dof_field[r], comp = L.dof_comp[r];
            const int64_t node = L.dof_node[r];
            int ne = 0;
            if (f < 2) {
                unflat(node, m2, dim, c);
                ne = touching_elements(c, 2, n, dim, els);
            } else {
                unflat(node, m1, dim, c);
                ne = touching_elements(c, 1, n, dim, els);
            }
            const bool solid_node = (f < 2) ? L.q2_solid[node] != 0 : false;
            for (int t = 0; t < ne; ++t) {
                const int64_t e = els[t];
                const bool se = L.material[e] != 0;
                const int32_t *ed = &L.elem_dofs[(size_t)e * nloc];
                auto add_range = [&](int lo, int hi) {
                    for (int q = lo; q < hi; ++q) cols.push_back(ed[q]);
                };
                const int D0 = 0, V0 = n2 * dim, P0 = 2 * n2 * dim;
                if (f == 0 && solid_node) {            // S row
                    if (se) {
                        add_range(D0, V0);
                        for (int b = 0; b < n2; ++b) cols.push_back(ed[V0 + b * dim + comp]);
                        add_range(P0, P0 + n1);
                    } else {
                        add_range(D0, P0 + n1);        // d, v and p^f of the fluid element
                    }
                } else if (f == 0) {                   // A row (fluid element only)
                    add_range(D0, V0);
                } else if (f == 1 && solid_node) {     // K row: lumped, diagonal per field
                    cols.push_back(L.d_dof[node * dim + comp]);
                    cols.push_back(L.v_dof[node * dim + comp]);
                    break;
                } else if (f == 1) {                   // F row
                    add_range(D0, P0 + n1);
                } else if (comp == 0) {                // V row (p^s): solid elements
                    if (se) {
                        add_range(D0, V0);
                        add_range(P0, P0 + n1);
                    }
                } else {                               // W row (p^f): fluid elements
                    if (!se) add_range(V0, P0);
                    // on the moving fluid element div_x u depends on d through F
                    if (!se && L.nl_pattern) add_range(D0, V0);
                }
            }
            std::vector<int32_t> out;
            out.reserve(cols.size());
            for (int32_t cc : cols)
                if (cc >= 0 && !L.fixed[cc]) out.push_back(cc);
            std::sort(out.begin(), out.end());
            out.erase(std::unique(out.begin(), out.end()), out.end());
            rows[r].swap(out);
        }
    }
    HostCSR &P = L.pattern;
    P.n_rows = P.n_cols = L.n_dofs;
    P.ptr.assign(L.n_dofs + 1, 0);
    for (int64_t r = 0; r < L.n_dofs; ++r) P.ptr[r + 1] = P.ptr[r] + (int64_t)rows[r].size();
    P.col.resize(P.ptr.back());
    for (int64_t r = 0; r < L.n_dofs; ++r)
        std::copy(rows[r].begin(), rows[r].end(), P.col.begin() + P.ptr[r]);
}

std::string build_levels(const ProblemDesc &p, std::vector<LevelHost> &levels) {
    if (p.dim != 2 && p.dim != 3) return "dim must be 2 or 3";
    if (p.n_levels < 1 || p.n_levels > 16) return "n_levels out of range";
    if (p.n_fine < 1 || (p.n_fine % (1 << (p.n_levels - 1))) != 0)
        return "n_fine must be divisible by 2^(n_levels-1)";
    if (p.bc_preset != 0 && p.bc_preset != 1) return "unknown bc_preset";
    if ((p.bc_preset == 0) != (p.dim == 2)) return "bc preset 0 is 2D, preset 1 is 3D";
    const int L = p.n_levels, dim = p.dim;
    levels.assign(L, LevelHost());
    std::vector<std::vector<uint8_t>> mats(L);
    mats[L - 1] = p.material;
    int64_t n = p.n_fine;
    for (int l = L - 1; l > 0; --l) {
        const int64_t nc = n / 2;
        mats[l - 1].assign(ipow(nc, dim), 0);
        int64_t c[3], f[3];
        for (int64_t e = 0; e < ipow(nc, dim); ++e) {
            unflat(e, nc, dim, c);
            uint8_t any = 0;
            for (int o = 0; o < (1 << dim); ++o) {
                for (int k = 0; k < dim; ++k) f[k] = 2 * c[k] + ((o >> k) & 1);
                any |= mats[l][toflat(f, n, dim)];
            }
            mats[l - 1][e] = any ? 1 : 0;
        }
        n = nc;
    }
    for (int l = 0; l < L; ++l) {
        LevelHost &lev = levels[l];
        lev.dim = dim;
        lev.n = p.n_fine >> (L - 1 - l);
        lev.material = mats[l];
        lev.nl_pattern = p.nonlinear != 0;
        fill_level(lev, p);
        build_pattern(lev);
    }
    return "";
}

void build_prolongation(const LevelHost &fine, const LevelHost &coarse, HostCSR &P) {
    const int dim = fine.dim;
    const int64_t nc = coarse.n, m2f = 2 * (int64_t)fine.n + 1, m2c = 2 * nc + 1;
    const int64_t m1f = (int64_t)fine.n + 1, m1c = nc + 1;
    std::vector<std::vector<std::pair<int32_t, double>>> rows(fine.n_dofs);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t y = 0; y < fine.nq2; ++y) {
        int64_t pos[3], el[3], cn[3];
        double w1[3][3], dd[3];
        unflat(y, m2f, dim, pos);
        for (int k = 0; k < dim; ++k) {
            el[k] = std::min(pos[k] / 4, nc - 1);          // a coarse element spans 4 fine Q2 steps
            q2_basis((double)(pos[k] - 4 * el[k]) / 4.0, w1[k], dd);
        }
        const int n2 = (int)ipow(3, dim);
        for (int aa = 0; aa < n2; ++aa) {
            int ai[3] = {aa % 3, (aa / 3) % 3, (aa / 9) % 3};
            double wt = 1.0;
            for (int k = 0; k < dim; ++k) wt *= w1[k][ai[k]];
            if (wt == 0.0) continue;
            for (int k = 0; k < dim; ++k) cn[k] = 2 * el[k] + ai[k];
            const int64_t Y = toflat(cn, m2c, dim);
            for (int i = 0; i < dim; ++i) {
                const int32_t rd = fine.d_dof[y * dim + i], cd = coarse.d_dof[Y * dim + i];
                if (!fine.fixed[rd] && !coarse.fixed[cd]) rows[rd].push_back({cd, wt});
                const int32_t rv = fine.v_dof[y * dim + i], cv = coarse.v_dof[Y * dim + i];
                if (!fine.fixed[rv] && !coarse.fixed[cv]) rows[rv].push_back({cv, wt});
            }
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t z = 0; z < fine.nq1; ++z) {
        int64_t pos[3], cand[8], ec[3], cn[3];
        unflat(z, m1f, dim, pos);
        const int nc_el = touching_elements(pos, 2, nc, dim, cand);  // coarse element spans 2 fine Q1 steps
        for (int copy = 0; copy < 2; ++copy) {
            const int32_t r = copy == 0 ? fine.ps_dof[z] : fine.pf_dof[z];
            if (r < 0) continue;
            const uint8_t want = copy == 0 ? 1 : 0;
            int64_t E = -1;
            for (int t = 0; t < nc_el; ++t)
                if (coarse.material[cand[t]] == want) { E = cand[t]; break; }
            if (E < 0) continue;                                    // p^f with no coarse fluid parent
            unflat(E, nc, dim, ec);
            const int n1 = 1 << dim;
            for (int al = 0; al < n1; ++al) {
                double wt = 1.0;
                for (int k = 0; k < dim; ++k) {
                    const double t = (double)(pos[k] - 2 * ec[k]) / 2.0;
                    wt *= ((al >> k) & 1) ? t : (1.0 - t);
                    cn[k] = ec[k] + ((al >> k) & 1);
                }
                if (wt == 0.0) continue;
                const int64_t Z = toflat(cn, m1c, dim);
                const int32_t cc = copy == 0 ? coarse.ps_dof[Z] : coarse.pf_dof[Z];
                rows[r].push_back({cc, wt});
            }
        }
    }
    P.n_rows = fine.n_dofs;
    P.n_cols = coarse.n_dofs;
    P.ptr.assign(P.n_rows + 1, 0);
    for (int64_t r = 0; r < P.n_rows; ++r) {
        auto &v = rows[r];
        std::sort(v.begin(), v.end());
        P.ptr[r + 1] = P.ptr[r] + (int64_t)v.size();
    }
    P.col.resize(P.ptr.back());
    P.val.resize(P.ptr.back());
    for (int64_t r = 0; r < P.n_rows; ++r)
        for (size_t k = 0; k < rows[r].size(); ++k) {
            P.col[P.ptr[r] + k] = rows[r][k].first;
            P.val[P.ptr[r] + k] = rows[r][k].second;
        }
}

void build_restriction(const HostCSR &P, const LevelHost &fine, const LevelHost &coarse,
                       bool classical, HostCSR &R) {
    // R_{l-1,l}: same-equation blocks P_gg^T, plus the S <- F block through
    // P_{u^f,u^s} (fine F residual on u^f -> coarse S row on the node's d^s).
    std::vector<std::vector<std::pair<int32_t, double>>> rows(coarse.n_dofs);
    for (int64_t r = 0; r < P.n_rows; ++r) {
        const int64_t gf = fine.group_of(r);
        for (int64_t k = P.ptr[r]; k < P.ptr[r + 1]; ++k) {
            const int32_t c = P.col[k];
            const int64_t gc = coarse.group_of(c);
            if (classical || gf == gc) rows[c].push_back({(int32_t)r, P.val[k]});
            if (!classical && gf == 4 && gc == 3) {
                const int32_t cd = coarse.d_dof[(int64_t)coarse.dof_node[c] * coarse.dim + coarse.dof_comp[c]];
                if (!coarse.fixed[cd]) rows[cd].push_back({(int32_t)r, P.val[k]});
            }
        }
    }
    R.n_rows = coarse.n_dofs;
    R.n_cols = fine.n_dofs;
    R.ptr.assign(R.n_rows + 1, 0);
    for (int64_t r = 0; r < R.n_rows; ++r) {
        std::sort(rows[r].begin(), rows[r].end());
        R.ptr[r + 1] = R.ptr[r] + (int64_t)rows[r].size();
    }
    R.col.resize(R.ptr.back());
    R.val.resize(R.ptr.back());
    for (int64_t r = 0; r < R.n_rows; ++r)
        for (size_t k = 0; k < rows[r].size(); ++k) {
            R.col[R.ptr[r] + k] = rows[r][k].first;
            R.val[R.ptr[r] + k] = rows[r][k].second;
        }
}

void build_blocks(const LevelHost &L, int b, std::vector<int64_t> &blk_ptr, std::vector<int32_t> &blk_idx,
                  bool monolithic, std::vector<int32_t> *tags) {
    const int dim = L.dim;
    const int64_t n = L.n, m1 = n + 1;
    const int64_t ng = (m1 + b - 1) / b;
    const int64_t n_groups = ipow(ng, dim);
    const int n2 = (int)ipow(3, dim);
    std::vector<std::vector<int32_t>> per(n_groups * 3);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t g = 0; g < n_groups; ++g) {
        int64_t gc[3], z[3], els[8], ec[3], c[3];
        unflat(g, ng, dim, gc);
        std::vector<int64_t> sol_el, flu_el;
        std::vector<int32_t> ps, pf;
        const int64_t cnt = ipow(b, dim);
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t r = t;
            bool inside = true;
            for (int k = 0; k < dim; ++k) {
                z[k] = gc[k] * b + r % b;
                r /= b;
                if (z[k] >= m1) inside = false;
            }
            if (!inside) continue;
            const int64_t zz = toflat(z, m1, dim);
            const int ne = touching_elements(z, 1, n, dim, els);
            if (L.ps_dof[zz] >= 0) {
                ps.push_back(L.ps_dof[zz]);
                for (int q = 0; q < ne; ++q)
                    if (L.material[els[q]]) sol_el.push_back(els[q]);
            }
            if (L.pf_dof[zz] >= 0) {
                pf.push_back(L.pf_dof[zz]);
                for (int q = 0; q < ne; ++q)
                    if (!L.material[els[q]]) flu_el.push_back(els[q]);
            }
        }
        auto nodes_of = [&](std::vector<int64_t> &els_v, std::vector<int64_t> &nodes) {
            std::sort(els_v.begin(), els_v.end());
            els_v.erase(std::unique(els_v.begin(), els_v.end()), els_v.end());
            for (int64_t e : els_v) {
                unflat(e, n, dim, ec);
                for (int aa = 0; aa < n2; ++aa) {
                    int64_t ai[3] = {aa % 3, (aa / 3) % 3, (aa / 9) % 3};
                    for (int k = 0; k < dim; ++k) c[k] = 2 * ec[k] + ai[k];
                    nodes.push_back(toflat(c, 2 * n + 1, dim));
                }
            }
        };
        std::vector<int64_t> sn, fn;
        nodes_of(sol_el, sn);
        nodes_of(flu_el, fn);
        auto finish = [&](std::vector<int32_t> &v) {
            std::vector<int32_t> out;
            for (int32_t d : v)
                if (d >= 0 && !L.fixed[d]) out.push_back(d);
            std::sort(out.begin(), out.end());
            out.erase(std::unique(out.begin(), out.end()), out.end());
            v.swap(out);
        };
        std::vector<int32_t> &S = per[g * 3 + 0], &Fd = per[g * 3 + 1], &Fu = per[g * 3 + 2];
        if (monolithic) {
            // AS: one block per group, every variable whose support meets the
            // support of the group's pressures (both materials' elements)
            std::vector<int64_t> all_el(sol_el);
            all_el.insert(all_el.end(), flu_el.begin(), flu_el.end());
            std::vector<int64_t> an;
            nodes_of(all_el, an);
            for (int64_t y : an)
                for (int i = 0; i < dim; ++i) {
                    S.push_back(L.d_dof[y * dim + i]);
                    S.push_back(L.v_dof[y * dim + i]);
                }
            S.insert(S.end(), ps.begin(), ps.end());
            S.insert(S.end(), pf.begin(), pf.end());
            finish(S);
            continue;
        }
        if (!sol_el.empty()) {
            for (int64_t y : sn)
                for (int i = 0; i < dim; ++i) S.push_back(L.d_dof[y * dim + i]);
            S.insert(S.end(), ps.begin(), ps.end());
            finish(S);
        }
        if (!flu_el.empty()) {
            for (int64_t y : fn) {
                if (L.q2_solid[y]) continue;
                for (int i = 0; i < dim; ++i) {
                    Fd.push_back(L.d_dof[y * dim + i]);
                    Fu.push_back(L.v_dof[y * dim + i]);
                }
            }
            Fu.insert(Fu.end(), pf.begin(), pf.end());
            finish(Fd);
            finish(Fu);
        }
    }
    blk_ptr.assign(1, 0);
    blk_idx.clear();
    if (tags) tags->clear();
    for (size_t q = 0; q < per.size(); ++q) {
        const auto &v = per[q];
        if (v.empty()) continue;
        blk_idx.insert(blk_idx.end(), v.begin(), v.end());
        blk_ptr.push_back((int64_t)blk_idx.size());
        if (tags) {
            tags->push_back((int32_t)(q / 3));   // vertex group
            tags->push_back((int32_t)(q % 3));   // kind: 0 solid, 1 fluid-d, 2 fluid-u
        }
    }
}

int colour_period(int b) { return b == 1 ? 4 : (b == 2 ? 3 : 2); }

void sweep_passes(const LevelHost &L, int b, const std::vector<int32_t> &tags, std::vector<int32_t> &pass) {
    const int dim = L.dim;
    const int64_t ng = (L.n + 1 + b - 1) / b;
    const int k = colour_period(b);
    const int nc = (int)ipow(k, dim);
    const size_t nb = tags.size() / 2;
    pass.resize(nb);
    for (size_t j = 0; j < nb; ++j) {
        int64_t gc[3];
        unflat(tags[2 * j], ng, dim, gc);
        int colour = 0, kp = 1;
        for (int a = 0; a < dim; ++a) {
            colour += (int)(gc[a] % k) * kp;
            kp *= k;
        }
        pass[j] = tags[2 * j + 1] * nc + colour;
    }
}

}  // namespace fsi
