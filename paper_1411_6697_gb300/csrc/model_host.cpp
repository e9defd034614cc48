// model_host.cpp -- host construction of the block form of M and M^-1.
//
// M is fixed before the main loop (Sec. II, Sec. V). Here it is built per
// parity sector from the orbit table and each sector block is inverted in
// long double; the composed inverse is then checked against the full 16x16 M
// with rows m_1..m_16 of Sec. II.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "model.h"

namespace lbk {

namespace {

// In-place Gauss-Jordan inverse of an n x n row-major block (n <= 4).
bool invert_block(const double* a, double* ainv, int n)
{
    long double m[4][8];
    long double scale = 0;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < 2 * n; c++) {
            m[r][c] = c < n ? (long double)a[r * n + c] : (long double)((c - n) == r);
            if (c < n && fabsl(m[r][c]) > scale) scale = fabsl(m[r][c]);
        }
    if (scale == 0) return false;
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabsl(m[r][col]) > fabsl(m[piv][col])) piv = r;
        if (fabsl(m[piv][col]) <= 1e-13L * scale) return false;
        for (int c = 0; c < 2 * n; c++) {
            long double t = m[col][c];
            m[col][c] = m[piv][c];
            m[piv][c] = t;
        }
        long double d = m[col][col];
        for (int c = 0; c < 2 * n; c++) m[col][c] /= d;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            long double f = m[r][col];
            for (int c = 0; c < 2 * n; c++) m[r][c] -= f * m[col][c];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) ainv[r * n + c] = (double)m[r][n + c];
    return true;
}

// velocity (vx, vy) of slot q of an orbit of the given kind and speed
void velocity(int kind, double c, int q, double* vx, double* vy)
{
    static const int ax[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const int dg[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    const int(*t)[2] = kind == 0 ? ax : dg;
    *vx = c * t[q][0];
    *vy = c * t[q][1];
}

// Apply the block inverse to a moment vector mh (standard order) -> f.
void apply_block_inverse(const HostModel& h, const double* mh, double* f)
{
    double es[4] = {mh[0], mh[3], mh[4] + mh[6], mh[13] + mh[15]};
    double ea[2] = {mh[4] - mh[6], mh[13] - mh[15]};
    double xo[4] = {mh[1], mh[7], mh[9], mh[11]};
    double yo[4] = {mh[2], mh[8], mh[12], mh[10]};
    double oo[2] = {mh[5], mh[14]};
    double pes[4], pea[2], px[4], py[4], po[2];
    for (int r = 0; r < 4; r++) {
        pes[r] = px[r] = py[r] = 0;
        for (int c = 0; c < 4; c++) {
            pes[r] += h.Ies[r * 4 + c] * es[c];
            px[r] += h.Iodd[r * 4 + c] * xo[c];
            py[r] += h.Iodd[r * 4 + c] * yo[c];
        }
    }
    for (int r = 0; r < 2; r++) {
        pea[r] = h.Iea[r * 2] * ea[0] + h.Iea[r * 2 + 1] * ea[1];
        po[r] = h.Ioo[r * 2] * oo[0] + h.Ioo[r * 2 + 1] * oo[1];
    }
    // axis orbits 0 (slot 0 of each sector) and 2 (slot 1)
    for (int a = 0; a < 2; a++) {
        double P = pes[a], Mm = pea[a], X = px[a], Y = py[a];
        double* g = f + 8 * a;
        g[0] = P + Mm + X;
        g[2] = P + Mm - X;
        g[1] = P - Mm + Y;
        g[3] = P - Mm - Y;
    }
    // diagonal orbits 1 (slot 2) and 3 (slot 3)
    for (int d = 0; d < 2; d++) {
        double e = pes[2 + d], X = px[2 + d], Y = py[2 + d], o = po[d];
        double* g = f + 4 + 8 * d;
        g[0] = e + X + Y + o;
        g[1] = e - X + Y - o;
        g[2] = e - X - Y + o;
        g[3] = e + X - Y - o;
    }
}

} // namespace

int build_host_model(const int32_t kind[4], const double speed[4], const double eta[4],
                     double gamma, HostModel* h, char* err, int errlen)
{
    memset(h, 0, sizeof(*h));
    if (!(kind[0] == 0 && kind[1] == 1 && kind[2] == 0 && kind[3] == 1)) {
        snprintf(err, errlen,
                 "orbit_kind must be {0,1,0,1}: two axis and two diagonal orbits are needed "
                 "for a non-singular M, taken in the order axis, diagonal, axis, diagonal");
        return -1;
    }
    h->I = 2.0 / (gamma - 1.0) - 2.0;
    for (int o = 0; o < 4; o++) {
        double c = speed[o];
        h->c[o] = c;
        h->w[o] = (kind[o] == 0 ? c * c : 2.0 * c * c) + eta[o] * eta[o];
    }
    const double *c = h->c, *w = h->w;
    double Bes[16] = {1.0,          1.0,          1.0,
                      1.0,          w[0],         w[2],
                      w[1],         w[3],         c[0] * c[0],
                      c[2] * c[2],  2 * c[1] * c[1], 2 * c[3] * c[3],
                      w[0] * c[0] * c[0], w[2] * c[2] * c[2], 2 * w[1] * c[1] * c[1],
                      2 * w[3] * c[3] * c[3]};
    double Bea[4] = {c[0] * c[0], c[2] * c[2], w[0] * c[0] * c[0], w[2] * c[2] * c[2]};
    double Bodd[16] = {c[0],        c[2],        c[1],        c[3],
                       w[0] * c[0], w[2] * c[2], w[1] * c[1], w[3] * c[3],
                       c[0] * c[0] * c[0], c[2] * c[2] * c[2], c[1] * c[1] * c[1],
                       c[3] * c[3] * c[3],
                       0.0,         0.0,         c[1] * c[1] * c[1], c[3] * c[3] * c[3]};
    double Boo[4] = {c[1] * c[1], c[3] * c[3], w[1] * c[1] * c[1], w[3] * c[3] * c[3]};
    memcpy(h->Bes, Bes, sizeof(Bes));
    memcpy(h->Bea, Bea, sizeof(Bea));
    memcpy(h->Bodd, Bodd, sizeof(Bodd));
    memcpy(h->Boo, Boo, sizeof(Boo));
    if (!invert_block(Bes, h->Ies, 4) || !invert_block(Bea, h->Iea, 2) ||
        !invert_block(Bodd, h->Iodd, 4) || !invert_block(Boo, h->Ioo, 2)) {
        snprintf(err, errlen, "singular moment matrix M for this velocity set");
        return -1;
    }
    // fold the butterfly scales into the inverse rows
    for (int k = 0; k < 16; k++) h->Ies[k] *= 0.25;
    for (int k = 0; k < 4; k++) h->Iea[k] *= 0.25, h->Ioo[k] *= 0.25;
    for (int r = 0; r < 4; r++)
        for (int k = 0; k < 4; k++) h->Iodd[r * 4 + k] *= (r < 2 ? 0.5 : 0.25);

    // full M in the standard row order, velocity order orbit-major
    for (int o = 0; o < 4; o++)
        for (int q = 0; q < 4; q++) {
            int i = 4 * o + q;
            double vx, vy;
            velocity(kind[o], speed[o], q, &vx, &vy);
            double ww = vx * vx + vy * vy + eta[o] * eta[o];
            double col[16] = {1.0,           vx,           vy,           ww,
                              vx * vx,       vx * vy,      vy * vy,      ww * vx,
                              ww * vy,       vx * vx * vx, vx * vx * vy, vx * vy * vy,
                              vy * vy * vy,  ww * vx * vx, ww * vx * vy, ww * vy * vy};
            for (int k = 0; k < 16; k++) h->M[k * 16 + i] = col[k];
        }
    // composed inverse, column by column, and its residual
    for (int k = 0; k < 16; k++) {
        double e[16] = {0}, f[16];
        e[k] = 1.0;
        apply_block_inverse(*h, e, f);
        for (int i = 0; i < 16; i++) h->Minv[i * 16 + k] = f[i];
    }
    double res = 0, mscale = 0;
    for (int r = 0; r < 16; r++)
        for (int cc = 0; cc < 16; cc++) {
            double s = 0;
            for (int k = 0; k < 16; k++) s += h->M[r * 16 + k] * h->Minv[k * 16 + cc];
            double d = fabs(s - (r == cc ? 1.0 : 0.0));
            if (d > res) res = d;
            if (fabs(h->M[r * 16 + cc]) > mscale) mscale = fabs(h->M[r * 16 + cc]);
        }
    h->residual = res;
    if (!(res < 1e-9)) {
        snprintf(err, errlen, "moment matrix M is numerically singular (|M Minv - 1| = %g)", res);
        return -1;
    }
    return 0;
}

template <typename R>
void fill_model_const(const HostModel& hm, const double S[16], double Q, double omega1,
                      double omega2, double T_ig, double dx, double dy, double dt, int nx,
                      int ny, int pitch, int bc_x, int bc_y, ModelConst<R>* K)
{
    memset(K, 0, sizeof(*K));
    for (int k = 0; k < 16; k++) {
        K->Bes[k] = (R)hm.Bes[k];
        K->Bodd[k] = (R)hm.Bodd[k];
        K->Ies[k] = (R)hm.Ies[k];
        K->Iodd[k] = (R)hm.Iodd[k];
        K->S[k] = (R)S[k];
    }
    for (int k = 0; k < 4; k++) {
        K->Bea[k] = (R)hm.Bea[k];
        K->Boo[k] = (R)hm.Boo[k];
        K->Iea[k] = (R)hm.Iea[k];
        K->Ioo[k] = (R)hm.Ioo[k];
        K->c[k] = (R)hm.c[k];
        K->cd[k] = hm.c[k];
        K->wd[k] = hm.w[k];
    }
    K->A8c = (R)((S[4] - S[7]) / S[4]);
    K->A9c = (R)((S[6] - S[8]) / S[6]);
    double DI = 2.0 + hm.I;
    K->DI = (R)DI;
    K->inv_DI = (R)(1.0 / DI);
    K->inv_DId = 1.0 / DI;
    K->omega1 = (R)omega1;
    K->omega2 = (R)omega2;
    K->chem = (R)(2.0 * Q / (DI * dt));
    K->dt = (R)dt;
    K->inv_dx = (R)(1.0 / dx);
    K->inv_dy = (R)(1.0 / dy);
    K->half_inv_dx = (R)(0.5 / dx);
    K->half_inv_dy = (R)(0.5 / dy);
    K->dx_ = (R)dx;
    K->T_igd = T_ig;
    auto split = [](double v, float& h, float& l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int k = 0; k < 4; k++) {
        split(K->cd[k], K->cdh[k], K->cdl[k]);
        split(K->wd[k], K->wdh[k], K->wdl[k]);
    }
    split(K->inv_DId, K->idh, K->idl);
    split(K->T_igd, K->tigh, K->tigl);
    K->nx = nx;
    K->ny = ny;
    K->pitch = pitch;
    K->bc_x = bc_x;
    K->bc_y = bc_y;
    K->plane = (int64_t)ny * pitch;
}

template void fill_model_const<float>(const HostModel&, const double*, double, double, double,
                                      double, double, double, double, int, int, int, int, int,
                                      ModelConst<float>*);
template void fill_model_const<double>(const HostModel&, const double*, double, double, double,
                                       double, double, double, double, int, int, int, int, int,
                                       ModelConst<double>*);

} // namespace lbk
