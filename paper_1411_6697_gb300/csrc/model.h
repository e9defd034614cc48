// model.h -- constants of the 16-velocity MRT-LBKM model as the kernels see them.
//
// The moment matrix M (rows m_1..m_16 of Sec. II, listed after Eq. (16)) is
// block-diagonal after a butterfly inside each orbit of four velocities:
//   axis orbit a (speed c, velocities (c,0),(0,c),(-c,0),(0,-c)):
//     sx = f0+f2, sy = f1+f3, P = sx+sy, Mm = sx-sy, ax = f0-f2, ay = f1-f3
//   diagonal orbit d (velocities (c,c),(-c,c),(-c,-c),(c,-c)):
//     e = f0+f1+f2+f3, ax = f0-f1-f2+f3, ay = f0+f1-f2-f3, o = f0-f1+f2-f3
// and the moments split by parity in (v_x, v_y):
//   ES: (P0, P2, e1, e3) -> (m1, m4, m5+m7, m14+m16)          4x4 "Bes"
//   EA: (Mm0, Mm2)       -> (m5-m7, m14-m16)                  2x2 "Bea"
//   OX: (ax0, ax2, ax1, ax3) -> (m2, m8, m10, m12)            4x4 "Bodd"
//   OY: (ay0, ay2, ay1, ay3) -> (m3, m9, m13, m11)            same Bodd
//   OO: (o1, o3)          -> (m6, m15)                        2x2 "Boo"
// (orbits 0, 2 are axis orbits, 1, 3 diagonal; w = v^2 + eta^2 of the orbit).
// The inverse blocks carry the butterfly scale factors (1/4 for P, Mm, e, ax/ay
// of diagonal orbits and o; 1/2 for ax/ay of axis orbits), so M^-1 is five
// small matrix products plus sums and differences. All of it is delivered to
// the kernels by value, i.e. through the constant bank of the launch.
#pragma once
#include <stdint.h>

namespace lbk {

constexpr int NV = 16;     // velocities = moments
constexpr int NPLANE = 17; // f_1..f_16 and lambda
constexpr int TNE_K = 12;  // Delta_5..Delta_16 (Delta_1..4 vanish)
// per-block TNE partial: sum[12], abs[12], min[12], max[12], d_sum, d2_sum
constexpr int TNE_PART = 4 * TNE_K + 2;

template <typename R>
struct ModelConst {
    R Bes[16], Bea[4], Bodd[16], Boo[4]; // forward blocks (row-major)
    R Ies[16], Iea[4], Iodd[16], Ioo[4]; // inverse blocks, butterfly scales folded
    R c[4];                              // orbit speeds
    R S[16];                             // relaxation rates R_1..R_16
    R A8c, A9c;                          // (S5-S8)/S5, (S7-S9)/S7 (Eqs. (3)-(4))
    R DI, inv_DI;                        // D + I and its inverse
    R omega1, omega2;                    // Cochran constants (Eq. (28))
    R chem;                              // 2 Q / ((D+I) dt): C_hat = dfeq/dT * dlambda * chem
    R dt, inv_dx, inv_dy, half_inv_dx, half_inv_dy, dx_;
    double cd[4], wd[4];                 // speeds and w in FP64 (conserved-moment recovery)
    double inv_DId, T_igd;
    // the same four FP64 quantities split as hi + lo FP32 pairs (double-float recovery)
    float cdh[4], cdl[4], wdh[4], wdl[4], idh, idl, tigh, tigl;
    R wux[2], wuy[2], wT[2];             // walls below row 0 [0] and above row ny-1 [1]
    int32_t sbc[4];                      // condition of the sides x=0, x=nx, y=0, y=ny:
                                         // 0 periodic, 1 zero gradient, 2 wall (y),
                                         // 3 Dirichlet, 4 specular (y)
    R sfeq[4][17];                       // Dirichlet ghost values (f_1..f_16, lambda)
    int32_t nx, ny, pitch, bc_x, bc_y;   // bc_y = 2: walls (non-equilibrium extrapolation)
    int32_t pad_;
    int64_t plane;                       // elements per plane = ny * pitch
};

struct HostModel {
    double Bes[16], Bea[4], Bodd[16], Boo[4];
    double Ies[16], Iea[4], Iodd[16], Ioo[4];
    double c[4], w[4], I;
    double M[256], Minv[256]; // full matrices (standard order) for checks
    double residual;          // max |M Minv - 1|
};

// Build the block form for the orbit table; returns 0, or -1 if a block is
// singular (message in err), checking the composed inverse against the full M.
int build_host_model(const int32_t kind[4], const double speed[4], const double eta[4],
                     double gamma, HostModel* out, char* err, int errlen);

template <typename R>
void fill_model_const(const HostModel& hm, const double S[16], double Q, double omega1,
                      double omega2, double T_ig, double dx, double dy, double dt, int nx,
                      int ny, int pitch, int bc_x, int bc_y, ModelConst<R>* K);

} // namespace lbk
