// Nonlinear monolithic FSI residual and its exact Newton Jacobian (Sec. 2.2),
// 2D, on the reference mesh of every level.
//
// Unknowns U = (d, u, p) in J2 order.  Per element (side h, 3-point Gauss
// rule per direction) the residual has three groups of rows (the J2 row of
// each local equation as in the linear assembly):
//   momentum (Eq. momentum_supg), test phi_a e_i, in the flux form
//       R_ai = sum_q dX [ A_i phi_a + sum_J B_iJ d_J phi_a / h ]
//     solid (total Lagrangian, Mooney-Rivlin sigma = -p I + 2 C1 (B - I)
//     - 2 C2 (B^{-1} - I), B = F F^T, F = I + grad_X d):
//       A_i = rho_s (u - u_n)_i / dt,
//       B = 1/2 (P(F) + P(F_n)) - p J F^{-T},  P(F) = J sigma_el F^{-T};
//     fluid (ALE on the current element, grad_x = F^{-T} grad_X, mesh
//     velocity w_m = (d - d_n)/dt, convecting velocity c = u - w_m):
//       A_i = rho J (u - u_n)_i / dt + 1/2 [J rho (c.grad_x u - f)_i + J_n rho (c_n.grad_x u_n - f_n)_i]
//       B_iJ = 1/2 [J (sigma F^{-T})_iJ + J_n (sigma_n F_n^{-T})_iJ] - J p F^{-1}_Ji
//              + J tau r_i rho (c F^{-T})_J          (SUPG, Eq. phi_SUPG)
//       with sigma = mu (grad_x u + grad_x u^T), c_n = u_n - w_m, and the
//       strong residual r = rho (u - u_n)/dt + rho c.grad_x u + grad_x p
//       - mu div_x(grad_x u + grad_x u^T) - rho f at the new state;
//   kinematic rows: solid K rows M_L (u - (d - d_n)/dt) (row-sum lumped mass),
//     fluid A rows k int (grad d + grad d^T) : grad phi_a (harmonic extension, k = 1/V_el fine);
//   continuity rows: solid V rows -int (J - 1) psi_b, fluid W rows -int J div_x u psi_b.
// tau (Eq. tausupg, Eq. lambda_k) = min(1/(4 lambda nu), 1/(sqrt(lambda) |u|)),
// lambda the largest eigenvalue of the bubble problem of the current element
// (its centre Q2 function, both components), from 50 steps of the power
// method started at (1, 1).  Crank-Nicolson for the spatial operator, a
// backward difference for the time derivatives, pressure at the new level.
//
// Jacobian: forward-mode dual numbers.  A thread owns one (element, local
// unknown t) pair and evaluates the element residual with the derivative
// seeded in unknown t, giving column t of the element Jacobian exactly (tau
// and its power iterations included).  The quantities interpolated at the
// quadrature points (values of d, u, p and their gradients and Hessians)
// are computed once per element and point into shared memory; each thread
// adds the derivative of its own seed.  Types are chosen per seed kind at
// compile time (d-, u- or p-seeded): quantities that do not depend on the
// seeded field stay plain doubles, so no derivative work is spent on them.
// Elements are processed in 4 colours (parity of the element coordinates):
// elements of one colour share no node, so the CSR values (or the residual
// vector) are accumulated without atomics, in a fixed order -- the assembly
// is bitwise repeatable.
#include <type_traits>

#include "context.h"

namespace fsi {

// element tables of the nonlinear level (2D): constant-memory Gauss tables
__constant__ double c_phi[9 * 9];        // [q][a]      Q2 values, x-fastest nodes and points
__constant__ double c_dphi[9 * 2 * 9];   // [q][J][a]   reference gradients
__constant__ double c_ddphi[9 * 3 * 9];  // [q][JK][a]  reference Hessian: xx, yy, xy
__constant__ double c_psi[9 * 4];        // [q][b]      Q1 values
__constant__ double c_dpsi[9 * 2 * 4];   // [q][J][b]   Q1 reference gradients
__constant__ double c_wq[9];             // weights on [0,1]^2
__constant__ double c_lump[9];           // int phi_a on [0,1]^2 (row-sum lumped mass / h^2)

namespace {

#define DEV __device__ __forceinline__

// ------------------------------------------------------------ dual numbers
struct Dl {
    double v, d;
    Dl() = default;
    __device__ __forceinline__ Dl(double x) : v(x), d(0.0) {}
    __device__ __forceinline__ Dl(double x, double dx) : v(x), d(dx) {}
};
DEV Dl operator+(Dl a, Dl b) { return {a.v + b.v, a.d + b.d}; }
DEV Dl operator+(Dl a, double b) { return {a.v + b, a.d}; }
DEV Dl operator+(double a, Dl b) { return {a + b.v, b.d}; }
DEV Dl operator-(Dl a, Dl b) { return {a.v - b.v, a.d - b.d}; }
DEV Dl operator-(Dl a, double b) { return {a.v - b, a.d}; }
DEV Dl operator-(double a, Dl b) { return {a - b.v, -b.d}; }
DEV Dl operator-(Dl a) { return {-a.v, -a.d}; }
DEV Dl operator*(Dl a, Dl b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
DEV Dl operator*(Dl a, double b) { return {a.v * b, a.d * b}; }
DEV Dl operator*(double a, Dl b) { return {a * b.v, a * b.d}; }
DEV Dl operator/(Dl a, Dl b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
DEV Dl operator/(double a, Dl b) {
    const double q = a / b.v;
    return {q, -q * b.d / b.v};
}
DEV Dl dsqrt(Dl a) {
    const double s = sqrt(a.v);
    return {s, 0.5 * a.d / s};
}
DEV double dsqrt(double a) { return sqrt(a); }
DEV double vpart(double a) { return a; }
DEV double vpart(Dl a) { return a.v; }

template <class T> struct is_dual : std::false_type {};
template <> struct is_dual<Dl> : std::true_type {};

template <class T> DEV T seeded(double v, double d) {
    if constexpr (is_dual<T>::value) return Dl{v, d};
    else return v;
}

// output of an expression: its value (residual) or its derivative (Jacobian)
template <bool JAC> DEV double ext(double a) { return JAC ? 0.0 : a; }
template <bool JAC> DEV double ext(Dl a) { return JAC ? a.d : a.v; }
// whether an expression of type T contributes to the output
template <bool JAC, class T> inline constexpr bool live = !JAC || is_dual<T>::value;

// types per seed kind: -1 none (residual), 0 a d unknown, 1 a u unknown, 2 a p unknown
template <int KIND> struct Ty {
    using D = std::conditional_t<KIND == 0, Dl, double>;
    using U = std::conditional_t<KIND == 1, Dl, double>;
    using P = std::conditional_t<KIND == 2, Dl, double>;
    using W = std::conditional_t<(KIND >= 0), Dl, double>;
};

// quantities interpolated at one quadrature point of one element
struct QV {
    double dq[2], gd[4], dnq[2];             // d, grad_X d (i-major: [i][J]); old d
    double uq[2], gu[4], hu[6], unq[2];      // u, grad_X u, Hessian [i][xx, yy, xy]; old u
    double pq, gp[2];                        // p, grad_X p
    double fn[2], fo[2];                     // body force at t_new and t_new - dt
    double J, Fi[4];                         // new state: det F, F^{-1} (row-major)
    double Jn, y[4];                         // old state: det F_n, grad_x u_n (fluid)
    double bo[4];                            // old-state part of B: solid 1/2 P_el(F_n),
                                             // fluid 1/2 J_n sigma_n F_n^{-T}
};

// gathered local values of one element
struct EV {
    double d[18], dn[18], u[18], un[18], p[4], w[18];
};

// shape tables addressed by a thread's own seed (node or vertex index
// differs across the warp): a shared-memory copy in the Jacobian kernels,
// the constant tables in the residual kernel (which has no seed)
struct Tab {
    const double *phi, *dphi, *ddphi, *psi, *dpsi;
};
constexpr int TAB_DOUBLES = 81 + 162 + 243 + 36 + 72;

struct NlArgs {
    int n;                      // elements per direction of the level
    double h, ih, dt, idt, rho_s, rho_f, mu_f, C1, C2, k_ale, fnew, fold;
    int32_t ds_end;             // dofs below: d^s (solid-class d)
    const int32_t *elem_dofs;   // n_el x 40: d(a,i), u(a,i), p(b)
    const uint8_t *material;
    const uint8_t *fixed;
    const double *w;            // 2 x nq2 level field of the body force
    const int32_t *elems;       // element list of the launch (one colour)
    int64_t n_elems;
    const double *U, *Un;
    // residual
    double *R;
    // Jacobian (CSR)
    const int32_t *row_ptr, *col;
    const int32_t *pos;         // n_el x 40 (local column) x 40 (local row): CSR position, -1 none, -2 absent
    double *val;
    int *err;
};

DEV void load_element(const NlArgs &A, int64_t e, EV &E) {
    const int32_t *ed = A.elem_dofs + e * 40;
    for (int k = 0; k < 18; ++k) {
        const int32_t cd = ed[k], cu = ed[18 + k];
        E.d[k] = A.U[cd];
        E.dn[k] = A.Un[cd];
        E.u[k] = A.U[cu];
        E.un[k] = A.Un[cu];
    }
    for (int b = 0; b < 4; ++b) E.p[b] = A.U[ed[36 + b]];
    const int64_t ex = e % A.n, ey = e / A.n, m2 = 2 * (int64_t)A.n + 1, nq2 = m2 * m2;
    for (int a = 0; a < 9; ++a) {
        const int64_t node = (2 * ey + a / 3) * m2 + 2 * ex + a % 3;
        E.w[2 * a] = A.w[node];
        E.w[2 * a + 1] = A.w[nq2 + node];
    }
}

// F = I + grad d, J = det F, Fi = F^{-1} (row-major 2 x 2)
template <class T>
DEV void kinematics(const T g[4], T &J, T Fi[4]) {
    const T F00 = 1.0 + g[0], F01 = g[1], F10 = g[2], F11 = 1.0 + g[3];
    J = F00 * F11 - F01 * F10;
    const T iJ = 1.0 / J;
    Fi[0] = F11 * iJ;
    Fi[1] = -F01 * iJ;
    Fi[2] = -F10 * iJ;
    Fi[3] = F00 * iJ;
}

// first Piola-Kirchhoff stress of the elastic part of the Mooney-Rivlin law:
// P = J sigma_el F^{-T}, sigma_el = 2 C1 (F F^T - I) - 2 C2 (F^{-T} F^{-1} - I)
template <class T>
DEV void piola_el(const T g[4], const T &J, const T Fi[4], double C1, double C2, T P[4]) {
    const T F00 = 1.0 + g[0], F01 = g[1], F10 = g[2], F11 = 1.0 + g[3];
    const T B00 = F00 * F00 + F01 * F01, B01 = F00 * F10 + F01 * F11, B11 = F10 * F10 + F11 * F11;
    const T Bi00 = Fi[0] * Fi[0] + Fi[2] * Fi[2], Bi01 = Fi[0] * Fi[1] + Fi[2] * Fi[3],
            Bi11 = Fi[1] * Fi[1] + Fi[3] * Fi[3];
    const T s00 = 2.0 * C1 * (B00 - 1.0) - 2.0 * C2 * (Bi00 - 1.0);
    const T s01 = 2.0 * C1 * B01 - 2.0 * C2 * Bi01;
    const T s11 = 2.0 * C1 * (B11 - 1.0) - 2.0 * C2 * (Bi11 - 1.0);
    // P_iK = J sum_j s_ij Fi_Kj
    P[0] = J * (s00 * Fi[0] + s01 * Fi[1]);
    P[1] = J * (s00 * Fi[2] + s01 * Fi[3]);
    P[2] = J * (s01 * Fi[0] + s11 * Fi[1]);
    P[3] = J * (s01 * Fi[2] + s11 * Fi[3]);
}

// Everything at quadrature point q of one element that does not depend on
// a seed: interpolated values, gradients and Hessians, the kinematics of the
// new and the old state and the old state's stress terms.
DEV void prepare_point(const NlArgs &A, const double *d, const double *dn, const double *u, const double *un,
                       const double *p, const double *w, bool solid, int q, QV &Q) {
    const double ih = A.ih, ih2 = A.ih * A.ih;
    double gdn[4], gun[4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        double s0 = 0, s1 = 0, s2 = 0, s3 = 0, g0 = 0, g1 = 0, gn0 = 0, gn1 = 0;
        double hu0 = 0, hu1 = 0, hu2 = 0, gu0 = 0, gu1 = 0, gun0 = 0, gun1 = 0, f = 0;
        for (int a = 0; a < 9; ++a) {
            const double ph = c_phi[q * 9 + a], dx = c_dphi[(q * 2) * 9 + a], dy = c_dphi[(q * 2 + 1) * 9 + a];
            const double da = d[2 * a + i], dna = dn[2 * a + i], ua = u[2 * a + i], una = un[2 * a + i];
            s0 += da * ph; s1 += dna * ph; s2 += ua * ph; s3 += una * ph;
            g0 += da * dx; g1 += da * dy; gn0 += dna * dx; gn1 += dna * dy;
            gu0 += ua * dx; gu1 += ua * dy; gun0 += una * dx; gun1 += una * dy;
            hu0 += ua * c_ddphi[(q * 3) * 9 + a];
            hu1 += ua * c_ddphi[(q * 3 + 1) * 9 + a];
            hu2 += ua * c_ddphi[(q * 3 + 2) * 9 + a];
            f += w[2 * a + i] * ph;
        }
        Q.dq[i] = s0; Q.dnq[i] = s1; Q.uq[i] = s2; Q.unq[i] = s3;
        Q.gd[2 * i] = g0 * ih; Q.gd[2 * i + 1] = g1 * ih;
        gdn[2 * i] = gn0 * ih; gdn[2 * i + 1] = gn1 * ih;
        Q.gu[2 * i] = gu0 * ih; Q.gu[2 * i + 1] = gu1 * ih;
        gun[2 * i] = gun0 * ih; gun[2 * i + 1] = gun1 * ih;
        Q.hu[3 * i] = hu0 * ih2; Q.hu[3 * i + 1] = hu1 * ih2; Q.hu[3 * i + 2] = hu2 * ih2;
        Q.fn[i] = A.fnew * f;
        Q.fo[i] = A.fold * f;
    }
    double pq = 0, gp0 = 0, gp1 = 0;
    for (int b = 0; b < 4; ++b) {
        pq += p[b] * c_psi[q * 4 + b];
        gp0 += p[b] * c_dpsi[(q * 2) * 4 + b];
        gp1 += p[b] * c_dpsi[(q * 2 + 1) * 4 + b];
    }
    Q.pq = pq;
    Q.gp[0] = gp0 * ih;
    Q.gp[1] = gp1 * ih;
    kinematics(Q.gd, Q.J, Q.Fi);
    double Fin[4];
    kinematics(gdn, Q.Jn, Fin);
    if (solid) {
        double Pn[4];
        piola_el(gdn, Q.Jn, Fin, A.C1, A.C2, Pn);
        for (int k = 0; k < 4; ++k) Q.bo[k] = 0.5 * Pn[k];
        for (int k = 0; k < 4; ++k) Q.y[k] = 0.0;
    } else {
        // grad_x u_n = grad_X u_n F_n^{-1}; sigma_n = mu (y + y^T); 1/2 J_n sigma_n F_n^{-T}
        const double y00 = gun[0] * Fin[0] + gun[1] * Fin[2], y01 = gun[0] * Fin[1] + gun[1] * Fin[3];
        const double y10 = gun[2] * Fin[0] + gun[3] * Fin[2], y11 = gun[2] * Fin[1] + gun[3] * Fin[3];
        Q.y[0] = y00; Q.y[1] = y01; Q.y[2] = y10; Q.y[3] = y11;
        const double mu = A.mu_f;
        const double t00 = 2.0 * mu * y00, t01 = mu * (y01 + y10), t11 = 2.0 * mu * y11;
        const double hj = 0.5 * Q.Jn;
        Q.bo[0] = hj * (t00 * Fin[0] + t01 * Fin[1]);
        Q.bo[1] = hj * (t00 * Fin[2] + t01 * Fin[3]);
        Q.bo[2] = hj * (t01 * Fin[0] + t11 * Fin[1]);
        Q.bo[3] = hj * (t01 * Fin[2] + t11 * Fin[3]);
    }
}

// grad_X d, J and F^{-1} at point q with the seed of a d unknown (node sa,
// component si): dF = e_si (x) grad_X phi_sa, dJ = J tr(F^{-1} dF),
// dF^{-1} = -F^{-1} dF F^{-1}; plain values for the other kinds
template <int KIND>
DEV void seeded_kin(const Tab &T, const QV &Q, int q, int sa, int si, double ih, typename Ty<KIND>::D g[4],
                    typename Ty<KIND>::D &J, typename Ty<KIND>::D Fi[4]) {
    if constexpr (KIND == 0) {
        const double g0 = T.dphi[(q * 2) * 9 + sa] * ih, g1 = T.dphi[(q * 2 + 1) * 9 + sa] * ih;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            g[2 * r] = Dl(Q.gd[2 * r], r == si ? g0 : 0.0);
            g[2 * r + 1] = Dl(Q.gd[2 * r + 1], r == si ? g1 : 0.0);
        }
        const double c0 = si ? Q.Fi[1] : Q.Fi[0], c1 = si ? Q.Fi[3] : Q.Fi[2];   // column si of F^{-1}
        J = Dl(Q.J, Q.J * (c0 * g0 + c1 * g1));
        const double v0 = g0 * Q.Fi[0] + g1 * Q.Fi[2], v1 = g0 * Q.Fi[1] + g1 * Q.Fi[3];
        Fi[0] = Dl(Q.Fi[0], -c0 * v0);
        Fi[1] = Dl(Q.Fi[1], -c0 * v1);
        Fi[2] = Dl(Q.Fi[2], -c1 * v0);
        Fi[3] = Dl(Q.Fi[3], -c1 * v1);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            g[k] = Q.gd[k];
            Fi[k] = Q.Fi[k];
        }
        J = Q.J;
    }
}

DEV double dabs(double a) { return fabs(a); }
DEV Dl dabs(Dl a) { return a.v < 0.0 ? -a : a; }

// symmetric 2 x 2 products (powers of one symmetric matrix commute)
template <class T> DEV void sym_mul(const T a[3], const T b[3], T c[3]) {
    const T c00 = a[0] * b[0] + a[1] * b[1], c01 = a[0] * b[1] + a[1] * b[2], c11 = a[1] * b[1] + a[2] * b[2];
    c[0] = c00; c[1] = c01; c[2] = c11;
}

// lambda_k of the element (bubble eigenproblem, power method)
template <int KIND, class GetQ>
DEV typename Ty<KIND>::D element_lambda(const NlArgs &A, const Tab &Tb, GetQ getQ, int sa, int si) {
    using TD = typename Ty<KIND>::D;
    const double ih = A.ih, ih2 = A.ih * A.ih, hh = A.h * A.h;
    TD K00 = 0.0, K01 = 0.0, K11 = 0.0, M = 0.0;
    for (int q = 0; q < 9; ++q) {
        const QV &Q = getQ(q);
        TD g[4], J, Fi[4];
        seeded_kin<KIND>(Tb, Q, q, sa, si, ih, g, J, Fi);
        // grad_x of the bubble (centre node 4) and its spatial Hessian Fi^T H Fi
        const double bx = c_dphi[(q * 2) * 9 + 4] * ih, by = c_dphi[(q * 2 + 1) * 9 + 4] * ih;
        const double Hxx = c_ddphi[(q * 3) * 9 + 4] * ih2, Hyy = c_ddphi[(q * 3 + 1) * 9 + 4] * ih2,
                     Hxy = c_ddphi[(q * 3 + 2) * 9 + 4] * ih2;
        const TD gb0 = bx * Fi[0] + by * Fi[2], gb1 = bx * Fi[1] + by * Fi[3];
        // T_Jk = sum_K H_JK Fi_Kk
        const TD T00 = Hxx * Fi[0] + Hxy * Fi[2], T01 = Hxx * Fi[1] + Hxy * Fi[3];
        const TD T10 = Hxy * Fi[0] + Hyy * Fi[2], T11 = Hxy * Fi[1] + Hyy * Fi[3];
        const TD H00 = Fi[0] * T00 + Fi[2] * T10, H01 = Fi[0] * T01 + Fi[2] * T11;
        const TD H11 = Fi[1] * T01 + Fi[3] * T11;
        const TD lap = H00 + H11;
        const TD wJ = (c_wq[q] * hh) * J;
        K00 = K00 + wJ * (lap * lap + 2.0 * lap * H00 + H00 * H00 + H01 * H01);
        K01 = K01 + wJ * (2.0 * lap * H01 + H00 * H01 + H01 * H11);
        K11 = K11 + wJ * (lap * lap + 2.0 * lap * H11 + H01 * H01 + H11 * H11);
        M = M + wJ * (gb0 * gb0 + gb1 * gb1);
    }
    // 50 power steps from (1, 1): the direction of K^50 (1, 1), formed by
    // squaring K / s (s >= |lambda|_max / 4 keeps every power in range; the
    // direction does not depend on the scale), K^50 = K^32 K^16 K^2
    const TD is = 1.0 / (dabs(K00) + dabs(K11) + 2.0 * dabs(K01));
    TD P1[3] = {K00 * is, K01 * is, K11 * is}, P2[3], P4[3], P8[3], P16[3], P32[3], T[3], P50[3];
    sym_mul(P1, P1, P2);
    sym_mul(P2, P2, P4);
    sym_mul(P4, P4, P8);
    sym_mul(P8, P8, P16);
    sym_mul(P16, P16, P32);
    sym_mul(P32, P16, T);
    sym_mul(T, P2, P50);
    const TD a0 = P50[0] + P50[1], a1 = P50[1] + P50[2];
    return (a0 * (K00 * a0 + K01 * a1) + a1 * (K01 * a0 + K11 * a1)) / (M * (a0 * a0 + a1 * a1));
}

// Element residual (JAC = false, KIND = -1) or column t of the element
// Jacobian (JAC = true, KIND = seed kind, t = local index within the kind).
// out[40] in the local row layout: momentum 0..17, kinematic 18..35,
// continuity 36..39.  For the Jacobian the lumped-mass entry of the solid
// K rows (row 18 + t of a d or u seed) is returned in *kin instead, so that
// out[] is only indexed by unrolled loop counters (it stays in registers).
template <int KIND, bool JAC, class GetQ>
DEV void element_rows(const NlArgs &A, const Tab &Tb, GetQ getQ, bool solid, int t, const EV *E, double *out,
                      double *kin) {
    using TD = typename Ty<KIND>::D;
    using TU = typename Ty<KIND>::U;
    using TP = typename Ty<KIND>::P;
    using TW = typename Ty<KIND>::W;
    const int sa = t >> 1, si = t & 1;
    const double ih = A.ih, ih2 = A.ih * A.ih, hh = A.h * A.h, idt = A.idt;
#pragma unroll
    for (int r = 0; r < 40; ++r) out[r] = 0.0;
    *kin = 0.0;
    if (solid) {   // kinematic K rows: lumped mass (u - (d - d_n)/dt)
        if constexpr (!JAC) {
#pragma unroll
            for (int k = 0; k < 18; ++k) out[18 + k] = hh * c_lump[k >> 1] * (E->u[k] - (E->d[k] - E->dn[k]) * idt);
        } else if constexpr (KIND == 0) {
            *kin = -hh * c_lump[sa] * idt;
        } else if constexpr (KIND == 1) {
            *kin = hh * c_lump[sa];
        }
    }
    // tau's element factors (Eq. tausupg): 1/(4 lambda nu) and 1/sqrt(lambda)
    TD t1 = 0.0, rsl = 0.0;
    if (!solid) {
        const TD lam = element_lambda<KIND>(A, Tb, getQ, sa, si);
        t1 = 1.0 / (4.0 * (A.mu_f / A.rho_f) * lam);
        rsl = 1.0 / dsqrt(lam);
    }
    for (int q = 0; q < 9; ++q) {
        const QV &Q = getQ(q);
        const double dX = c_wq[q] * hh;
        TD g[4], J, Fi[4];
        seeded_kin<KIND>(Tb, Q, q, sa, si, ih, g, J, Fi);
        const double Jn = Q.Jn;
        const TP p = seeded<TP>(Q.pq, KIND == 2 ? Tb.psi[q * 4 + (t & 3)] : 0.0);
        TU uq[2];
        for (int i = 0; i < 2; ++i) uq[i] = seeded<TU>(Q.uq[i], si == i ? Tb.phi[q * 9 + sa] : 0.0);
        TW Ai[2], B[4], C;
        if (solid) {
            TD P[4];
            piola_el(g, J, Fi, A.C1, A.C2, P);
            for (int i = 0; i < 2; ++i) {
                Ai[i] = A.rho_s * (uq[i] - Q.unq[i]) * idt;
                for (int K = 0; K < 2; ++K) B[2 * i + K] = 0.5 * P[2 * i + K] + Q.bo[2 * i + K] - p * J * Fi[2 * K + i];
            }
            C = -(J - 1.0);
        } else {
            TD dq[2], wm[2];
            for (int i = 0; i < 2; ++i) {
                dq[i] = seeded<TD>(Q.dq[i], si == i ? Tb.phi[q * 9 + sa] : 0.0);
                wm[i] = (dq[i] - Q.dnq[i]) * idt;
            }
            TU gu[4], hu[6];
            for (int i = 0; i < 2; ++i) {
                for (int Jd = 0; Jd < 2; ++Jd)
                    gu[2 * i + Jd] = seeded<TU>(Q.gu[2 * i + Jd], si == i ? Tb.dphi[(q * 2 + Jd) * 9 + sa] * ih : 0.0);
                for (int k = 0; k < 3; ++k)
                    hu[3 * i + k] = seeded<TU>(Q.hu[3 * i + k], si == i ? Tb.ddphi[(q * 3 + k) * 9 + sa] * ih2 : 0.0);
            }
            // new state: grad_x u = grad_X u F^{-1}
            const auto x00 = gu[0] * Fi[0] + gu[1] * Fi[2], x01 = gu[0] * Fi[1] + gu[1] * Fi[3];
            const auto x10 = gu[2] * Fi[0] + gu[3] * Fi[2], x11 = gu[2] * Fi[1] + gu[3] * Fi[3];
            const auto c0 = uq[0] - wm[0], c1 = uq[1] - wm[1];
            const auto cv0 = c0 * x00 + c1 * x01, cv1 = c0 * x10 + c1 * x11;
            const double mu = A.mu_f, rho = A.rho_f;
            const auto s00 = 2.0 * mu * x00, s01 = mu * (x01 + x10), s11 = 2.0 * mu * x11;
            // old state (its mesh velocity is the new one)
            const auto n0 = Q.unq[0] - wm[0], n1 = Q.unq[1] - wm[1];
            const auto cn0 = n0 * Q.y[0] + n1 * Q.y[1], cn1 = n0 * Q.y[2] + n1 * Q.y[3];
            // SUPG: strong residual at the new state
            const TU Hx0[3] = {hu[0], hu[1], hu[2]}, Hx1[3] = {hu[3], hu[4], hu[5]};
            // spatial Hessian of u_i: Fi^T H Fi ([jk]: 00, 11, 01)
            auto push = [&](const TU *Hr, auto &o00, auto &o11, auto &o01) {
                const auto T00 = Hr[0] * Fi[0] + Hr[2] * Fi[2], T01 = Hr[0] * Fi[1] + Hr[2] * Fi[3];
                const auto T10 = Hr[2] * Fi[0] + Hr[1] * Fi[2], T11 = Hr[2] * Fi[1] + Hr[1] * Fi[3];
                o00 = Fi[0] * T00 + Fi[2] * T10;
                o01 = Fi[0] * T01 + Fi[2] * T11;
                o11 = Fi[1] * T01 + Fi[3] * T11;
            };
            decltype(Hx0[0] * Fi[0]) a00, a11, a01, b00, b11, b01;
            push(Hx0, a00, a11, a01);
            push(Hx1, b00, b11, b01);
            // div_x (grad_x u + grad_x u^T): i = 0: 2 u0,xx + u0,yy + u1,xy; i = 1: u1,xx + 2 u1,yy + u0,xy
            const auto visc0 = 2.0 * a00 + a11 + b01, visc1 = b00 + 2.0 * b11 + a01;
            const TP gpr0 = seeded<TP>(Q.gp[0], KIND == 2 ? Tb.dpsi[(q * 2) * 4 + (t & 3)] * ih : 0.0);
            const TP gpr1 = seeded<TP>(Q.gp[1], KIND == 2 ? Tb.dpsi[(q * 2 + 1) * 4 + (t & 3)] * ih : 0.0);
            const auto gp0 = gpr0 * Fi[0] + gpr1 * Fi[2], gp1 = gpr0 * Fi[1] + gpr1 * Fi[3];
            const auto r0 = rho * (uq[0] - Q.unq[0]) * idt + rho * cv0 + gp0 - mu * visc0 - rho * Q.fn[0];
            const auto r1 = rho * (uq[1] - Q.unq[1]) * idt + rho * cv1 + gp1 - mu * visc1 - rho * Q.fn[1];
            // tau (Eq. tausupg): min(1/(4 lambda nu), 1/(sqrt(lambda) |u|))
            TW tau = t1;
            const auto sp2 = uq[0] * uq[0] + uq[1] * uq[1];
            if (vpart(sp2) > 0.0) {
                const TW t2 = rsl * (1.0 / dsqrt(sp2));
                if (vpart(t2) < vpart(tau)) tau = t2;
            }
            // convecting direction pulled back: c_J = rho sum_j c_j Fi_Jj
            const auto k0 = rho * (c0 * Fi[0] + c1 * Fi[1]), k1 = rho * (c0 * Fi[2] + c1 * Fi[3]);
            const auto Jt = J * tau;
            Ai[0] = rho * J * (uq[0] - Q.unq[0]) * idt + 0.5 * (J * rho * (cv0 - Q.fn[0]) + Jn * rho * (cn0 - Q.fo[0]));
            Ai[1] = rho * J * (uq[1] - Q.unq[1]) * idt + 0.5 * (J * rho * (cv1 - Q.fn[1]) + Jn * rho * (cn1 - Q.fo[1]));
            // B_iJ = 1/2 (J sigma Fi^T + J_n sigma_n Fi_n^T)_iJ - J p Fi_Ji + J tau r_i c_J
            const auto hJ = 0.5 * J;
            B[0] = hJ * (s00 * Fi[0] + s01 * Fi[1]) + Q.bo[0] - J * p * Fi[0] + Jt * r0 * k0;
            B[1] = hJ * (s00 * Fi[2] + s01 * Fi[3]) + Q.bo[1] - J * p * Fi[2] + Jt * r0 * k1;
            B[2] = hJ * (s01 * Fi[0] + s11 * Fi[1]) + Q.bo[2] - J * p * Fi[1] + Jt * r1 * k0;
            B[3] = hJ * (s01 * Fi[2] + s11 * Fi[3]) + Q.bo[3] - J * p * Fi[3] + Jt * r1 * k1;
            C = -J * (x00 + x11);
            // harmonic extension rows: k (grad d + grad d^T)
            if constexpr (live<JAC, TD>) {
                const double kk = A.k_ale * dX * ih;
                const TD G00 = 2.0 * g[0], G01 = g[1] + g[2], G11 = 2.0 * g[3];
                const double e00 = ext<JAC>(G00), e01 = ext<JAC>(G01), e11 = ext<JAC>(G11);
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const double dx = c_dphi[(q * 2) * 9 + a], dy = c_dphi[(q * 2 + 1) * 9 + a];
                    out[18 + 2 * a] += kk * (e00 * dx + e01 * dy);
                    out[18 + 2 * a + 1] += kk * (e01 * dx + e11 * dy);
                }
            }
        }
        const double A0 = ext<JAC>(Ai[0]), A1 = ext<JAC>(Ai[1]);
        const double B00 = ext<JAC>(B[0]) * ih, B01 = ext<JAC>(B[1]) * ih, B10 = ext<JAC>(B[2]) * ih,
                     B11 = ext<JAC>(B[3]) * ih;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double ph = c_phi[q * 9 + a], dx = c_dphi[(q * 2) * 9 + a], dy = c_dphi[(q * 2 + 1) * 9 + a];
            out[2 * a] += dX * (A0 * ph + B00 * dx + B01 * dy);
            out[2 * a + 1] += dX * (A1 * ph + B10 * dx + B11 * dy);
        }
        const double Cq = dX * ext<JAC>(C);
#pragma unroll
        for (int b = 0; b < 4; ++b) out[36 + b] += Cq * c_psi[q * 4 + b];
    }
}

// global row of local equation r of an element (-1: not assembled there)
DEV int32_t local_row(const int32_t *ed, bool solid, int32_t ds_end, int r) {
    if (r >= 36) return ed[r];
    const int k = r < 18 ? r : r - 18;
    const bool snode = ed[(k >> 1) * 2] < ds_end;      // d dof of the node is in d^s
    if (r < 18) return (solid || snode) ? ed[k] : ed[18 + k];   // momentum: S or F row
    if (solid) return ed[18 + k];                              // K row
    return snode ? -1 : ed[k];                                 // A row (fluid-class node)
}

DEV int find_col(const int32_t *col, int lo, int hi, int c) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// residual: one thread per element of the colour
__global__ void __launch_bounds__(128) nl_residual_kernel(NlArgs A) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= A.n_elems) return;
    const int64_t e = A.elems[k];
    EV E;
    load_element(A, e, E);
    const bool solid = A.material[e] != 0;
    QV Qs;
    auto getQ = [&](int q) -> const QV & {
        prepare_point(A, E.d, E.dn, E.u, E.un, E.p, E.w, solid, q, Qs);
        return Qs;
    };
    double out[40], kin;
    const Tab Tb{c_phi, c_dphi, c_ddphi, c_psi, c_dpsi};
    element_rows<-1, false>(A, Tb, getQ, solid, 0, &E, out, &kin);
    const int32_t *ed = A.elem_dofs + e * 40;
#pragma unroll
    for (int r = 0; r < 40; ++r) {
        const int32_t R = local_row(ed, solid, A.ds_end, r);
        if (R >= 0 && !A.fixed[R]) A.R[R] += out[r];
    }
}

// Point data of every element of a level (the seed-independent part of the
// Jacobian): a CTA gathers the local values of 8 elements into shared
// memory, then one thread per (element, point) writes its QV record to
// pts[(e * 9 + q)].  Run once per assembly and level, read by all three
// seed kinds.
constexpr int PT_EPB = 8;
__global__ void __launch_bounds__(PT_EPB * 9) nl_point_kernel(NlArgs A, int64_t n_el, QV *pts) {
    __shared__ double s_ev[PT_EPB][94];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * PT_EPB;
    for (int k = tid; k < PT_EPB * 94; k += PT_EPB * 9) {
        const int el = k / 94, j = k % 94;
        const int64_t e = base + el;
        if (e >= n_el) continue;
        const int32_t *ed = A.elem_dofs + e * 40;
        double v;
        if (j < 18) v = A.U[ed[j]];
        else if (j < 36) v = A.Un[ed[j - 18]];
        else if (j < 54) v = A.U[ed[j - 36 + 18]];
        else if (j < 72) v = A.Un[ed[j - 54 + 18]];
        else if (j < 76) v = A.U[ed[36 + j - 72]];
        else {
            const int a = (j - 76) >> 1, i = (j - 76) & 1;
            const int64_t ex = e % A.n, ey = e / A.n, m2 = 2 * (int64_t)A.n + 1;
            v = A.w[i * m2 * m2 + (2 * ey + a / 3) * m2 + 2 * ex + a % 3];
        }
        s_ev[el][j] = v;
    }
    __syncthreads();
    const int el = tid / 9, q = tid % 9;
    const int64_t e = base + el;
    if (e >= n_el) return;
    const double *v = s_ev[el];
    QV Q;
    prepare_point(A, v, v + 18, v + 36, v + 54, v + 72, v + 76, A.material[e] != 0, q, Q);
    pts[e * 9 + q] = Q;
}

// Jacobian: EPB elements per CTA, NT threads per element (18 for d and u
// seeds, 4 for p seeds); the elements' point records are copied from the
// point scratch into shared memory, then every thread evaluates one column
// of an element Jacobian and adds it into the CSR values.
template <int KIND, int EPB, int NT, int MINB>
__global__ void __launch_bounds__(EPB *NT, MINB) nl_jacobian_kernel(NlArgs A, const QV *__restrict__ pts) {
    __shared__ QV s_q[EPB][9];
    __shared__ double s_tab[TAB_DOUBLES];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * EPB;
    constexpr int QD = sizeof(QV) / sizeof(double);
    for (int k = tid; k < TAB_DOUBLES; k += EPB * NT)
        s_tab[k] = k < 81 ? c_phi[k]
                          : (k < 243 ? c_dphi[k - 81]
                                     : (k < 486 ? c_ddphi[k - 243] : (k < 522 ? c_psi[k - 486] : c_dpsi[k - 522])));
    double *sq = reinterpret_cast<double *>(&s_q[0][0]);
    for (int k = tid; k < EPB * 9 * QD; k += EPB * NT) {
        const int el = k / (9 * QD), r = k % (9 * QD);
        if (base + el >= A.n_elems) continue;
        const int64_t e = A.elems[base + el];
        sq[k] = reinterpret_cast<const double *>(pts + e * 9)[r];
    }
    __syncthreads();
    const int el = tid / NT, t = tid % NT;
    if (base + el >= A.n_elems) return;
    const int64_t e = A.elems[base + el];
    const bool solid = A.material[e] != 0;
    auto getQ = [&](int q) -> const QV & { return s_q[el][q]; };
    const Tab Tb{s_tab, s_tab + 81, s_tab + 243, s_tab + 486, s_tab + 522};
    double out[40], kin;
    element_rows<KIND, true>(A, Tb, getQ, solid, t, nullptr, out, &kin);
    const int lc = KIND == 0 ? t : (KIND == 1 ? 18 + t : 36 + t);
    const int4 *pp = reinterpret_cast<const int4 *>(A.pos + (e * 40 + lc) * 40);
#pragma unroll
    for (int r4 = 0; r4 < 10; ++r4) {
        const int4 p4 = pp[r4];
        const int pr[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = 4 * r4 + u;
            const double v = out[r] + (r == 18 + t ? kin : 0.0);
            if (v == 0.0 || pr[u] == -1) continue;   // structural zero, or a row/column not assembled
            if (pr[u] < 0) {                         // a coupling outside the operator pattern
                atomicOr(A.err, 1);
                continue;
            }
            A.val[pr[u]] += v;
        }
    }
}

// CSR position of every (local row, local column) pair of every element:
// -1 where the pair is not assembled (no row there, fixed row or column),
// -2 where the operator pattern lacks the pair (an error if a nonzero lands there)
__global__ void nl_pos_kernel(const int32_t *elem_dofs, const uint8_t *material, const uint8_t *fixed,
                              int32_t ds_end, const int32_t *row_ptr, const int32_t *col, int64_t n_el,
                              int32_t *pos) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_el * 40;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / 40;
        const int lc = (int)(k % 40);
        const int32_t *ed = elem_dofs + e * 40;
        const bool solid = material[e] != 0;
        const int32_t C = ed[lc];
        int32_t *out = pos + k * 40;
        for (int r = 0; r < 40; ++r) {
            const int32_t R = local_row(ed, solid, ds_end, r);
            if (R < 0 || fixed[R] || fixed[C]) {
                out[r] = -1;
                continue;
            }
            const int p = find_col(col, row_ptr[R], row_ptr[R + 1], C);
            out[r] = p >= 0 ? p : -2;
        }
    }
}

__global__ void nl_fixed_rows_kernel(const uint8_t *fixed, const double *U, double *R, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (fixed[i]) R[i] = U[i];
}

__global__ void nl_inject_kernel(const int32_t *map, const uint8_t *fixed, const double *Uf, double *Uc, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t m = map[i];
        Uc[i] = (m >= 0 && !fixed[i]) ? Uf[m] : 0.0;
    }
}

__global__ void nl_axpby_kernel(double *y, const double *x, double a, double b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

inline unsigned grid_of(int64_t n, int t) {
    int64_t g = (n + t - 1) / t;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

NlArgs make_args(const NlLevelDev &L, const NlParams &P, const double *U, const double *Un, double t_new) {
    NlArgs A{};
    A.n = L.n;
    A.h = 1.0 / L.n;
    A.ih = (double)L.n;
    A.dt = P.dt;
    A.idt = 1.0 / P.dt;
    A.rho_s = P.rho_s;
    A.rho_f = P.rho_f;
    A.mu_f = P.mu_f;
    A.C1 = P.C1;
    A.C2 = P.C2;
    A.k_ale = P.k_ale;
    const double two_pi = 6.283185307179586;
    A.fnew = P.force * sin(two_pi * t_new / P.period);
    A.fold = P.force * sin(two_pi * (t_new - P.dt) / P.period);
    A.ds_end = L.ds_end;
    A.elem_dofs = L.elem_dofs.as<int32_t>();
    A.material = L.material.as<uint8_t>();
    A.w = L.w.as<double>();
    A.U = U;
    A.Un = Un;
    return A;
}

}  // namespace

fsi_status nl_upload_tables(cudaStream_t s) {
    // 3-point Gauss-Legendre rule on [0, 1]; Q2 Lagrange polynomials on the
    // nodes 0, 1/2, 1 and their first and second derivatives; Q1 on 0, 1
    const double r = std::sqrt(0.6);
    const double gx[3] = {0.5 - 0.5 * r, 0.5, 0.5 + 0.5 * r};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    double v[3][3], dv[3][3], ddv[3], l1[3][2], dl1[2] = {-1.0, 1.0};
    ddv[0] = 4.0; ddv[1] = -8.0; ddv[2] = 4.0;
    for (int k = 0; k < 3; ++k) {
        const double x = gx[k];
        v[k][0] = 2.0 * (x - 0.5) * (x - 1.0);
        v[k][1] = -4.0 * x * (x - 1.0);
        v[k][2] = 2.0 * x * (x - 0.5);
        dv[k][0] = 4.0 * x - 3.0;
        dv[k][1] = 4.0 - 8.0 * x;
        dv[k][2] = 4.0 * x - 1.0;
        l1[k][0] = 1.0 - x;
        l1[k][1] = x;
    }
    double phi[81], dphi[162], ddphi[243], psi[36], dpsi[72], wq[9], lump[9];
    for (int a = 0; a < 9; ++a) lump[a] = 0.0;
    for (int qy = 0; qy < 3; ++qy)
        for (int qx = 0; qx < 3; ++qx) {
            const int q = qx + 3 * qy;
            wq[q] = gw[qx] * gw[qy];
            for (int ay = 0; ay < 3; ++ay)
                for (int ax = 0; ax < 3; ++ax) {
                    const int a = ax + 3 * ay;
                    phi[q * 9 + a] = v[qx][ax] * v[qy][ay];
                    dphi[(q * 2) * 9 + a] = dv[qx][ax] * v[qy][ay];
                    dphi[(q * 2 + 1) * 9 + a] = v[qx][ax] * dv[qy][ay];
                    ddphi[(q * 3) * 9 + a] = ddv[ax] * v[qy][ay];
                    ddphi[(q * 3 + 1) * 9 + a] = v[qx][ax] * ddv[ay];
                    ddphi[(q * 3 + 2) * 9 + a] = dv[qx][ax] * dv[qy][ay];
                    lump[a] += wq[q] * phi[q * 9 + a];
                }
            for (int by = 0; by < 2; ++by)
                for (int bx = 0; bx < 2; ++bx) {
                    const int b = bx + 2 * by;
                    psi[q * 4 + b] = l1[qx][bx] * l1[qy][by];
                    dpsi[(q * 2) * 4 + b] = dl1[bx] * l1[qy][by];
                    dpsi[(q * 2 + 1) * 4 + b] = l1[qx][bx] * dl1[by];
                }
        }
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_phi, phi, sizeof(phi), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_dphi, dphi, sizeof(dphi), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_ddphi, ddphi, sizeof(ddphi), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_psi, psi, sizeof(psi), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_dpsi, dpsi, sizeof(dpsi), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_wq, wq, sizeof(wq), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyToSymbolAsync(c_lump, lump, sizeof(lump), 0, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return FSI_OK;
}

fsi_status launch_nl_residual(const NlLevelDev &L, const NlParams &P, const uint8_t *fixed, int64_t n_dofs,
                              const double *U, const double *Un, double t_new, double *R, cudaStream_t s) {
    FSI_CUDA(cudaMemsetAsync(R, 0, (size_t)n_dofs * 8, s));
    NlArgs A = make_args(L, P, U, Un, t_new);
    A.fixed = fixed;
    A.R = R;
    for (int c = 0; c < 4; ++c) {
        const int64_t ne = L.colour_ptr[c + 1] - L.colour_ptr[c];
        if (ne == 0) continue;
        A.elems = L.elems.as<int32_t>() + L.colour_ptr[c];
        A.n_elems = ne;
        nl_residual_kernel<<<(unsigned)((ne + 127) / 128), 128, 0, s>>>(A);
        count_launch();
        FSI_CUDA(cudaGetLastError());
    }
    nl_fixed_rows_kernel<<<grid_of(n_dofs, 256), 256, 0, s>>>(fixed, U, R, n_dofs);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status nl_point_bytes(const NlLevelDev &L, size_t *bytes) {
    *bytes = (size_t)L.n * L.n * 9 * sizeof(QV);
    return FSI_OK;
}

fsi_status launch_nl_jacobian(const NlLevelDev &L, const NlParams &P, const uint8_t *fixed, const DevCSR &Aop,
                              const double *U, const double *Un, double t_new, int *err, cudaStream_t s,
                              ForkJoin *fj) {
    FSI_CUDA(cudaMemsetAsync(Aop.val64.p, 0, (size_t)Aop.nnz * 8, s));
    NlArgs A = make_args(L, P, U, Un, t_new);
    A.fixed = fixed;
    A.row_ptr = Aop.ptr.as<int32_t>();
    A.col = Aop.col.as<int32_t>();
    A.val = Aop.val64.as<double>();
    A.err = err;
    A.pos = L.pos.as<int32_t>();
    const int64_t n_el = (int64_t)L.n * L.n;
    if (!A.pos || L.pos.bytes < (size_t)n_el * 1600 * 4) { set_error("nonlinear position table missing"); return FSI_ERR_STATE; }
    QV *pts = L.pts.as<QV>();
    if (!pts || L.pts.bytes < (size_t)n_el * 9 * sizeof(QV)) { set_error("nonlinear point scratch missing"); return FSI_ERR_STATE; }
    nl_point_kernel<<<(unsigned)((n_el + PT_EPB - 1) / PT_EPB), PT_EPB * 9, 0, s>>>(A, n_el, pts);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    // the three seed kinds write disjoint columns: side by side on two
    // auxiliary streams; colours (which share rows) one after another
    constexpr int EPB = 8;
    for (int c = 0; c < 4; ++c) {
        const int64_t ne = L.colour_ptr[c + 1] - L.colour_ptr[c];
        if (ne == 0) continue;
        A.elems = L.elems.as<int32_t>() + L.colour_ptr[c];
        A.n_elems = ne;
        const unsigned g = (unsigned)((ne + EPB - 1) / EPB);
        for (int k = 0; k < 2; ++k) {
            FSI_CUDA(cudaEventRecord(fj[k].fork, s));
            FSI_CUDA(cudaStreamWaitEvent(fj[k].aux, fj[k].fork, 0));
        }
        nl_jacobian_kernel<0, EPB, 18, 2><<<g, EPB * 18, 0, s>>>(A, pts);
        nl_jacobian_kernel<1, EPB, 18, 1><<<g, EPB * 18, 0, fj[0].aux>>>(A, pts);
        nl_jacobian_kernel<2, EPB, 4, 1><<<g, EPB * 4, 0, fj[1].aux>>>(A, pts);
        count_launch(3);
        FSI_CUDA(cudaGetLastError());
        for (int k = 0; k < 2; ++k) {
            FSI_CUDA(cudaEventRecord(fj[k].join, fj[k].aux));
            FSI_CUDA(cudaStreamWaitEvent(s, fj[k].join, 0));
        }
    }
    FSI_TRY(launch_set_fixed_diag(Aop, fixed, Aop.val64.as<double>(), s));
    return FSI_OK;
}

fsi_status launch_nl_positions(NlLevelDev &L, const DevCSR &Aop, const uint8_t *fixed, cudaStream_t s) {
    const int64_t n_el = (int64_t)L.n * L.n;
    FSI_TRY(L.pos.alloc((size_t)n_el * 1600 * 4));
    nl_pos_kernel<<<grid_of(n_el * 40, 256), 256, 0, s>>>(L.elem_dofs.as<int32_t>(), L.material.as<uint8_t>(), fixed,
                                                           L.ds_end, Aop.ptr.as<int32_t>(), Aop.col.as<int32_t>(), n_el,
                                                           L.pos.as<int32_t>());
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_nl_axpby(double *y, const double *x, double a, double b, int64_t n, cudaStream_t s) {
    nl_axpby_kernel<<<grid_of(n, 256), 256, 0, s>>>(y, x, a, b, n);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

fsi_status launch_nl_inject(const int32_t *map, const uint8_t *fixed_c, const double *Uf, double *Uc, int64_t nc,
                            cudaStream_t s) {
    nl_inject_kernel<<<grid_of(nc, 256), 256, 0, s>>>(map, fixed_c, Uf, Uc, nc);
    count_launch();
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
}

}  // namespace fsi
