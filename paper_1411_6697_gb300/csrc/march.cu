// march.cu -- the FP32 2-D step kernel: y-marching strips, two cells per thread.
//
// A block of 64 threads owns a strip of 128 columns x `strip_rows` rows and
// marches up it one row per iteration. Thread t updates the cells (x0+2t, y)
// and (x0+2t+1, y) together, so most arithmetic runs as packed FP32 pairs
// (FFMA2 / FADD2 / FMUL2, sm_100+).
//
// Shared memory keeps the staged rows (128 + 4 columns, filled by 16- and 8-byte
// cp.async copies) of the 17 planes in rings sized by what each plane still
// needs: the y-stencil of a plane with v_y > 0 reads rows y-2..y+1, with v_y < 0
// rows y-1..y+2, with v_y = 0 only row y, lambda rows y-2..y+2; every plane also
// holds row y+2 (recovered this iteration) and the prefetched row y+3. That is
// 88 staged plane-rows instead of 17 x 7, which lets four blocks share an SM.
// A ring of 4 macro rows holds rho, u, T of rows y-1..y+2 (with one halo column
// on each side for grad u). Per iteration: wait for row y+2, one __syncthreads,
// issue the copy of row y+3, recover rho, u, T of row y+2 from its conserved
// moments, update row y. The
// conserved moments are summed exactly (TwoSum butterflies, split constants);
// rho, u, T are then formed in FP64 (REC = 0) or in double-float on the FP32
// pipes (REC = 1), and the ignition test T > T_ig is taken in that precision.
// The TNE statistics of the updated state's input (Delta_5..Delta_16, Sec. VI)
// accumulate in registers and are reduced per strip into FP64.
#include <float.h>
#include <stdlib.h>

#include "cell.cuh"
#include "kernels.cuh"
#include "pair.cuh"
#include "reduce.cuh"
#include "vec2.cuh"

namespace lbk {

namespace {

constexpr int MT = 64;         // threads per block
constexpr int NWM = MT / 32;   // warps per block
constexpr int BW = 2 * MT;     // columns per strip
constexpr int RW = BW + 4;     // staged row: x0-2 .. x0+BW+1
constexpr int PF = 1;          // staged rows in flight beyond y+2
constexpr int MRING = 4;       // macro rows kept
constexpr int MW = BW + 4;     // macro row: x0-2 .. x0+BW+1, own cells at even offsets

// plane classes by the sign of v_y (orbits 0 and 2 are axis orbits, 1 and 3
// diagonal): rows kept = rows the y-stencil reads below y+2, plus y+2 and y+3
enum { C_UP = 0, C_DN = 1, C_FLAT = 2, C_LAM = 3 };
constexpr int NROWS[4] = {6, 5, 4, 6};   // y-2..y+3, y-1..y+3, y..y+3, y-2..y+3
constexpr int NPL[4] = {6, 6, 4, 1};     // planes per class
__host__ __device__ constexpr int pclass(int p)
{
    return p == 16 ? C_LAM
                   : ((p & 3) == 0 || (p & 3) == 2) && ((p >> 2) & 1) == 0
                         ? C_FLAT
                         : (((p >> 2) & 1) == 0 ? ((p & 3) == 1 ? C_UP : C_DN)
                                                 : ((p & 3) < 2 ? C_UP : C_DN));
}
// index of plane p within its class, planes in increasing order (o = orbit,
// k = velocity within the orbit)
__host__ __device__ constexpr int pindex(int p)
{
    const int o = p >> 2, k = p & 3;
    return p == 16 ? 0
                   : pclass(p) == C_FLAT ? (o >> 1) * 2 + (k >> 1)
                                         : (o >> 1) * 3 + ((o & 1) ? (pclass(p) == C_UP ? 1 + k : k - 1) : 0);
}
__host__ __device__ constexpr bool class_layout_ok()
{
    int seen[4][8] = {};
    for (int p = 0; p < NPLANE; p++) {
        const int c = pclass(p), i = pindex(p);
        if (i < 0 || i >= NPL[c] || seen[c][i]) return false;
        seen[c][i] = 1;
    }
    return true;
}
static_assert(class_layout_ok(), "every plane has its own slot in its class");

// ring base (floats) of each class; the whole ring starts 2 floats into shared
// memory so that every row base is 2 mod 4 floats and column x0 (element 2 of a
// staged row) sits on a 16-byte boundary
constexpr int CBASE0 = 2;
constexpr int CBASE1 = CBASE0 + NROWS[0] * NPL[0] * RW;
constexpr int CBASE2 = CBASE1 + NROWS[1] * NPL[1] * RW;
constexpr int CBASE3 = CBASE2 + NROWS[2] * NPL[2] * RW;
constexpr int RING_FLOATS = CBASE3 + NROWS[3] * NPL[3] * RW;
static_assert(RW % 4 == 0 && CBASE1 % 4 == 2 && CBASE2 % 4 == 2 && CBASE3 % 4 == 2,
              "row bases must be 2 mod 4 floats");
static_assert(pclass(1) == C_UP && pclass(3) == C_DN && pclass(0) == C_FLAT && pclass(2) == C_FLAT &&
                  pclass(4) == C_UP && pclass(5) == C_UP && pclass(6) == C_DN && pclass(7) == C_DN &&
                  pclass(8) == C_FLAT && pclass(9) == C_UP && pclass(11) == C_DN &&
                  pclass(13) == C_UP && pclass(14) == C_DN && pindex(15) == 5 && pindex(10) == 3,
              "plane classes follow the orbit layout axis, diagonal, axis, diagonal");

constexpr size_t OFF_MAC = ((size_t)RING_FLOATS * 4 + 15) / 16 * 16;
constexpr size_t OFF_IGN = OFF_MAC + (size_t)4 * MRING * MW * 4;
constexpr size_t OFF_TSUM = (OFF_IGN + (size_t)MRING * BW + 15) / 16 * 16;
constexpr size_t OFF_TMM = OFF_TSUM + (size_t)NWM * NSUM * 8;
constexpr size_t MARCH_SMEM = OFF_TMM + (size_t)NWM * NMM * 4;
static_assert(MARCH_SMEM <= 56 * 1024, "four blocks per SM need <= 56 KB each");

__device__ __forceinline__ int mac_slot(int r) { return (r + MRING) & (MRING - 1); }

// start of the staged row r of class c
template <int CL>
__device__ __forceinline__ float* class_row(float* ring, int r)
{
    constexpr int N = NROWS[CL], np = NPL[CL];
    constexpr int base = CL == 0 ? CBASE0 : CL == 1 ? CBASE1 : CL == 2 ? CBASE2 : CBASE3;
    return ring + base + ((r + 8 * N) % N) * np * RW;
}
// the staged row r of plane p (p a compile-time constant after unrolling)
__device__ __forceinline__ float* plane_row(float* ring, int p, int r)
{
    const int c = pclass(p);
    float* b = c == C_UP ? class_row<C_UP>(ring, r)
                         : c == C_DN ? class_row<C_DN>(ring, r)
                                     : c == C_FLAT ? class_row<C_FLAT>(ring, r) : class_row<C_LAM>(ring, r);
    return b + pindex(p) * RW;
}

__device__ __forceinline__ void cp8(void* dst, const void* src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}

// n staged values of plane p, row r, columns x .. x+n-1 through the boundary rules
// (the rare path of the staging)
__device__ __forceinline__ void stage_elements(const ModelConst<float>& K, const float* in, float* dst,
                                            int p, int x, int r, int n)
{
    for (int e = 0; e < n; e++) dst[e] = ghost_value(K, in, p, x + e, r);
}

// Stage row r of the planes whose class is in `mask`, columns x0-2 .. x0+BW+1: the
// 32 16-byte chunks of columns x0 .. x0+BW-1 of a plane by one warp (lane = chunk),
// the two 8-byte edges (x0-2, x0-1 and x0+BW, x0+BW+1) of all planes by the first 34
// threads. Rows outside the grid follow the side's condition: a Dirichlet side fills
// the row with its equilibrium, a specular side copies the mirror row with the planes
// of reversed v_y, the others copy the wrapped or edge row (walls are corrected after
// the row lands). Columns outside the grid go element by element through the same
// rules (ghost_value).
template <bool GEN>
__device__ __forceinline__ void issue_row(const float* __restrict__ in, float* ring, int r,
                                          int x0, const ModelConst<float>& K, unsigned mask)
{
    static_assert(BW == 128 && NWM == 2, "staging layout assumes 32 chunks per row and 2 warps");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (!GEN) { // periodic or zero-gradient sides only: index maps, no ghost rules
        const float* rowp = in + (int64_t)map_index(r, K.ny, K.bc_y) * K.pitch;
#pragma unroll
        for (int p = 0; p < NPLANE; p++) {
            if ((p & 1) != w || !((mask >> pclass(p)) & 1u)) continue;
            float* dst = plane_row(ring, p, r) + 2 + 4 * lane;
            const float* src = rowp + p * K.plane;
            const int x = x0 + 4 * lane;
            if (x + 4 <= K.nx) {
                cp16(dst, src + x);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) dst[e] = src[map_index(x + e, K.nx, K.bc_x)];
            }
        }
        if (threadIdx.x < 2 * NPLANE) {
            const int p = threadIdx.x >> 1, side = threadIdx.x & 1;
            if ((mask >> pclass(p)) & 1u) {
                float* dst = plane_row(ring, p, r) + (side ? BW + 2 : 0);
                const float* src = rowp + p * K.plane;
                const int x = side ? x0 + BW : x0 - 2;
                if (x >= 0 && x + 2 <= K.nx) {
                    cp8(dst, src + x);
                } else {
                    dst[0] = src[map_index(x, K.nx, K.bc_x)];
                    dst[1] = src[map_index(x + 1, K.nx, K.bc_x)];
                }
            }
        }
        return;
    }
    int gy = r, dir_side = -1;
    bool mir = false;
    if (r < 0 || r >= K.ny) {
        const int s = r < 0 ? 2 : 3, code = K.sbc[s];
        if (code == 3) {
            dir_side = s;
        } else if (code == 4) {
            gy = r < 0 ? -r - 1 : 2 * K.ny - 1 - r;
            gy = gy < 0 ? 0 : (gy >= K.ny ? K.ny - 1 : gy);
            mir = true;
        } else {
            gy = map_index(r, K.ny, code == 0 ? 0 : 1);
        }
    }
    const float* rowp = in + (int64_t)gy * K.pitch;
#pragma unroll
    for (int p = 0; p < NPLANE; p++) {
        if ((p & 1) != w || !((mask >> pclass(p)) & 1u)) continue;
        float* dst = plane_row(ring, p, r) + 2 + 4 * lane;
        const int x = x0 + 4 * lane;
        if (dir_side >= 0) {
            const float v = K.sfeq[dir_side][p];
            *reinterpret_cast<float4*>(dst) = make_float4(v, v, v, v);
            continue;
        }
        const int sp = mir ? mirror_plane(p) : p;
        const float* src = rowp + sp * K.plane;
        if (x + 4 <= K.nx)
            cp16(dst, src + x);
        else
            stage_elements(K, in, dst, p, x, r, 4);
    }
    if (threadIdx.x < 2 * NPLANE) {
        const int p = threadIdx.x >> 1, side = threadIdx.x & 1;
        if ((mask >> pclass(p)) & 1u) {
            float* dst = plane_row(ring, p, r) + (side ? BW + 2 : 0);
            const int x = side ? x0 + BW : x0 - 2;
            if (dir_side < 0 && x >= 0 && x + 2 <= K.nx)
                cp8(dst, rowp + (mir ? mirror_plane(p) : p) * K.plane + x);
            else
                stage_elements(K, in, dst, p, x, r, 2);
        }
    }
}
constexpr unsigned ALL_CLASSES = 0xfu;

// Walls (Sec. IV.D): the staged ghost row r_ghost holds a copy of the fluid row r_src
// (the index map clamps); add the non-equilibrium-extrapolation correction to the
// thread's own two columns of the f planes that keep that row (only the v_y > 0
// class keeps row y0-2). Ghost rows are read only at the own columns of the thread
// that corrects them (y-stencils and macros), so no barrier follows.
__device__ __forceinline__ void wall_fix_row(float* ring, int r_ghost, int r_src, int side,
                                             const ModelConst<float>& K, bool up_only)
{
    const int lx = 2 * threadIdx.x + 2;
    V2 f[16], d[16];
#pragma unroll
    for (int i = 0; i < 16; i++) f[i] = ldv(plane_row(ring, i, r_src) + lx);
    wall_correction(K, f, side, d);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (up_only && pclass(i) != C_UP) continue;
        float* q = plane_row(ring, i, r_ghost) + lx;
        *reinterpret_cast<float2*>(q) = (ldv(q) + d[i]).v;
    }
}

struct MacRow {
    V2 rho, ux, uy, T;
    bool ig0, ig1;
    float hu, hv; // velocity of the halo column (threads 0 and MT-1)
};

// rho, u, T of the thread's two cells of staged row r, kept in registers until
// store_macros so that the update of an earlier row can run in between.
template <int REC>
__device__ __forceinline__ MacRow row_macros(const float* ring, int r, const ModelConst<float>& K,
                                             const DfConst& C, int& bad, bool act0, bool act1)
{
    const int tid = threadIdx.x;
    float* rg = const_cast<float*>(ring);
    const int lx = 2 * tid + 2;
    V2 f[16];
#pragma unroll
    for (int i = 0; i < 16; i++) f[i] = V2(*reinterpret_cast<const float2*>(plane_row(rg, i, r) + lx));
    MacRow o;
    bool ok0, ok1;
    recover_pair<REC>(f, C, K, o.rho, o.ux, o.uy, o.T, o.ig0, o.ig1, ok0, ok1);
    if ((act0 && !ok0) || (act1 && !ok1)) bad = 1;
    o.hu = o.hv = 0.f;
    if (tid == 0 || tid == MT - 1) { // halo columns x0-1 and x0+BW: velocity only
        const int hx = tid == 0 ? 1 : BW + 2;
        float g[16];
#pragma unroll
        for (int i = 0; i < 16; i++) g[i] = plane_row(rg, i, r)[hx];
        velocity_f32(g, K, o.hu, o.hv);
    }
    return o;
}

__device__ __forceinline__ void store_macros(float* mac, unsigned char* ign, int r, const MacRow& o)
{
    const int tid = threadIdx.x;
    const int ms = mac_slot(r);
    const int mi = 2 * tid + 2;
    *reinterpret_cast<float2*>(mac + (0 * MRING + ms) * MW + mi) = o.rho.v;
    *reinterpret_cast<float2*>(mac + (1 * MRING + ms) * MW + mi) = o.ux.v;
    *reinterpret_cast<float2*>(mac + (2 * MRING + ms) * MW + mi) = o.uy.v;
    *reinterpret_cast<float2*>(mac + (3 * MRING + ms) * MW + mi) = o.T.v;
    ign[ms * BW + 2 * tid] = o.ig0;
    ign[ms * BW + 2 * tid + 1] = o.ig1;
    if (tid == 0 || tid == MT - 1) {
        const int hm = tid == 0 ? 1 : BW + 2;
        mac[(1 * MRING + ms) * MW + hm] = o.hu;
        mac[(2 * MRING + ms) * MW + hm] = o.hv;
    }
}

template <int REC, bool GEN, bool AVG>
__global__ void __launch_bounds__(MT, 4)
    march_kernel(const ModelConst<float> K, const StepLaunch a, int strip_rows)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float* ring = reinterpret_cast<float*>(smem);  // class rings from float 2 on (see CBASE0)
    float* mac = reinterpret_cast<float*>(smem + OFF_MAC);
    unsigned char* ign = smem + OFF_IGN;
    double* tsum = reinterpret_cast<double*>(smem + OFF_TSUM);
    float* tmm = reinterpret_cast<float*>(smem + OFF_TMM);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = K.nx, ny = K.ny;
    const float* __restrict__ in = static_cast<const float*>(a.in);
    float* out = static_cast<float*>(a.out); // not restrict: prev may alias it
    // AVG: a later SSP Runge-Kutta stage, out = wp * u^n + wn * E(in), u^n read from prev
    // at the cell's own position (prev may be out itself: each value is read before it
    // is written, by the same thread)
    const float* pv = static_cast<const float*>(a.prev);
    const float wp = (float)a.wprev, wn = (float)a.wnew;

    const DfConst C = df_constants(K);

    const int64_t step = a.ctr->step;
    // AVG stages reduce no TNE
    const bool do_tne = !AVG && a.tne_every > 0 && (step % a.tne_every) == 0;
    if (do_tne) {
        for (int i = tid; i < NWM * NSUM; i += MT) tsum[i] = 0.0;
        for (int i = tid; i < NWM * NMM; i += MT) tmm[i] = (i % NMM) < TNE_K ? FLT_MAX : -FLT_MAX;
    }
    float tmin[TNE_K], tmax[TNE_K];
#pragma unroll
    for (int k = 0; k < TNE_K; k++) tmin[k] = FLT_MAX, tmax[k] = -FLT_MAX;
    int bad = 0;

    const int nsx = (nx + BW - 1) / BW, nsy = (ny + strip_rows - 1) / strip_rows;
    const int nstrips = nsx * nsy;
    const int lx = 2 * tid + 2;  // own cells in a staged row
    const int mi = 2 * tid + 2;  // own cells in a macro row
    const float dt = K.dt;

    for (int s = blockIdx.x; s < nstrips; s += gridDim.x) {
        const int x0 = (s / nsy) * BW, y0 = (s % nsy) * strip_rows;
        const int yend = y0 + strip_rows < ny ? y0 + strip_rows : ny;
        const int cx = x0 + 2 * tid;
        const bool act0 = cx < nx, act1 = cx + 1 < nx;
        float tsm[NSUM];
        V2 tsp[TNE_K], td2(0.f);
#pragma unroll
        for (int q = 0; q < NSUM; q++) tsm[q] = 0.f;
#pragma unroll
        for (int k = 0; k < TNE_K; k++) tsp[k] = V2(0.f);

        __syncthreads(); // the previous strip is done with the rings
        // rows y0-2 .. y0+2: row y0-2 only for the classes whose stencil reaches it
        for (int r = y0 - 2; r <= y0 + 1 + PF; r++) {
            if (r <= yend + 1)
                issue_row<GEN>(in, ring, r, x0, K,
                               r == y0 - 2 ? ((1u << C_UP) | (1u << C_LAM)) : ALL_CLASSES);
            cp_commit();
        }
        cp_wait<PF>(); // rows y0-2 .. y0+1 have landed
        __syncthreads();
        // walls: ghost rows among those landed (row y0+2 is fixed in the loop)
        if constexpr (GEN) {
            if (K.sbc[2] == 2) {
                if (y0 - 1 < 0) wall_fix_row(ring, y0 - 1, 0, 0, K, false);
                if (y0 - 2 < 0) wall_fix_row(ring, y0 - 2, 0, 0, K, true); // v_y > 0 only
            }
            if (K.sbc[3] == 2 && y0 + 1 >= ny) wall_fix_row(ring, y0 + 1, ny - 1, 1, K, false);
        }
        for (int r = y0 - 1; r <= y0 + 1; r++)
            store_macros(mac, ign, r, row_macros<REC>(ring, r, K, C, bad, act0, act1));

        for (int y = y0; y < yend; y++) {
            cp_wait<PF - 1>(); // row y+2 has landed
            __syncthreads();
            if (y + 2 + PF <= yend + 1) issue_row<GEN>(in, ring, y + 2 + PF, x0, K, ALL_CLASSES);
            cp_commit();
            if constexpr (GEN)
                if (K.sbc[3] == 2 && y + 2 >= ny) wall_fix_row(ring, y + 2, ny - 1, 1, K, false);
            // macros of row y+2 (read from the next iteration on)
            store_macros(mac, ign, y + 2, row_macros<REC>(ring, y + 2, K, C, bad, act0, act1));

            // ---------------- update of row y ----------------
            // row y of every plane; rows y-2..y+1 of the v_y > 0 class, y-1..y+2 of the
            // v_y < 0 class, y-2..y+2 of lambda
            const float* up_m2 = class_row<C_UP>(ring, y - 2);
            const float* up_m1 = class_row<C_UP>(ring, y - 1);
            const float* up_p1 = class_row<C_UP>(ring, y + 1);
            const float* dn_m1 = class_row<C_DN>(ring, y - 1);
            const float* dn_p1 = class_row<C_DN>(ring, y + 1);
            const float* dn_p2 = class_row<C_DN>(ring, y + 2);
            const float* lm = class_row<C_LAM>(ring, y);
            const int ms = mac_slot(y), msm = mac_slot(y - 1), msp = mac_slot(y + 1);
            V2 f[16];
#pragma unroll
            for (int i = 0; i < 16; i++) f[i] = ldv(plane_row(ring, i, y) + lx);
            const V2 lam0 = ldv(lm + lx);
            const V2 rho = ldv(mac + (0 * MRING + ms) * MW + mi);
            const V2 ux = ldv(mac + (1 * MRING + ms) * MW + mi);
            const V2 uy = ldv(mac + (2 * MRING + ms) * MW + mi);
            const V2 T = ldv(mac + (3 * MRING + ms) * MW + mi);
            const bool ig0 = ign[ms * BW + 2 * tid], ig1 = ign[ms * BW + 2 * tid + 1];

            // moments, equilibrium, non-equilibrium parts
            V2 m[16], q[16], D[TNE_K];
            forward_moments(K, f, m);
            feq_moments(V2(K.DI), rho, ux, uy, T, q);
#pragma unroll
            for (int k = 0; k < TNE_K; k++) D[k] = m[k + 4] - q[k + 4];

            // grad u: x from the macro row (halo columns included), y from rows y+-1
            const float* uxr = mac + (1 * MRING + ms) * MW;
            const float* uyr = mac + (2 * MRING + ms) * MW;
            const float2 uxl = *reinterpret_cast<const float2*>(uxr + mi - 2);
            const float2 uxh = *reinterpret_cast<const float2*>(uxr + mi + 2);
            const float2 uyl = *reinterpret_cast<const float2*>(uyr + mi - 2);
            const float2 uyh = *reinterpret_cast<const float2*>(uyr + mi + 2);
            const V2 dux_dx = (V2(ux.y(), uxh.x) - V2(uxl.y, ux.x())) * K.half_inv_dx;
            const V2 duy_dx = (V2(uy.y(), uyh.x) - V2(uyl.y, uy.x())) * K.half_inv_dx;
            const V2 dux_dy = (ldv(mac + (1 * MRING + msp) * MW + mi) -
                               ldv(mac + (1 * MRING + msm) * MW + mi)) * K.half_inv_dy;
            const V2 duy_dy = (ldv(mac + (2 * MRING + msp) * MW + mi) -
                               ldv(mac + (2 * MRING + msm) * MW + mi)) * K.half_inv_dy;
            const V2 theta = (dux_dx + duy_dy) * K.inv_DI;
            const V2 shear = duy_dx + dux_dy;
            const V2 rT = rho * T;
            const V2 A8 = (rT * K.A8c) * fma(V2(4.f) * ux, dux_dx - theta, V2(2.f) * uy * shear);
            const V2 A9 = (rT * K.A9c) * fma(V2(4.f) * uy, duy_dy - theta, V2(2.f) * ux * shear);

            // reaction over dt (Eq. (28)), decided by the recovered T
            // (evaluated for both cells and selected: no divergent branch)
            const float ri0 = reaction_increment(lam0.x(), K.omega1 * rT.x(), K.omega2 * rT.x(), dt);
            const float ri1 = reaction_increment(lam0.y(), K.omega1 * rT.y(), K.omega2 * rT.y(), dt);
            const float dl0 = ig0 ? ri0 : 0.f, dl1 = ig1 ? ri1 : 0.f;
            const V2 dlam(dl0, dl1);
            const V2 cr = dlam * K.chem;

            // collision in moment space and back
            V2 dq[16], Om[16], W[16];
            dfeq_dT(V2(K.DI), rho, ux, uy, T, dq);
            Om[0] = Om[1] = Om[2] = V2(0.f);
            Om[3] = dq[3] * cr;
#pragma unroll
            for (int k = 4; k < 16; k++) Om[k] = fma(V2(-K.S[k]), D[k - 4], dq[k] * cr);
            Om[7] += A8;
            Om[8] += A9;
            inverse_moments(K, Om, W);

            // lambda: u . grad(lambda) with NND interface values
            const Q6 lq = load6(lm, lx);
            const float* lm_m2 = class_row<C_LAM>(ring, y - 2);
            const float* lm_m1 = class_row<C_LAM>(ring, y - 1);
            const float* lm_p1 = class_row<C_LAM>(ring, y + 1);
            const float* lm_p2 = class_row<C_LAM>(ring, y + 2);
            const V2 lpx = nnd_pos_x(lq), lnx = nnd_neg_x(lq);
            const V2 lpy = nnd_pos_y(ldv(lm_m2 + lx), ldv(lm_m1 + lx), lam0, ldv(lm_p1 + lx));
            const V2 lny = nnd_neg_y(ldv(lm_m1 + lx), lam0, ldv(lm_p1 + lx), ldv(lm_p2 + lx));
            const V2 lax(ux.x() > 0.f ? lpx.x() : lnx.x(), ux.y() > 0.f ? lpx.y() : lnx.y());
            const V2 lay(uy.x() > 0.f ? lpy.x() : lny.x(), uy.y() > 0.f ? lpy.y() : lny.y());
            const V2 ladv = fma(ux * K.inv_dx, lax, uy * K.inv_dy * lay);
            V2 ln = fma(V2(-dt), ladv, lam0) + dlam;
            ln = vmin(vmax(ln, V2(0.f)), V2(1.f));

            // NND flux differences (upwind side fixed per velocity), Euler update, store
            const int64_t g = (int64_t)y * K.pitch + cx;
            auto put = [&](int i, V2 adv) {
                V2 v = fma(V2(dt), W[i] - adv, f[i]);
                if (act1) {
                    float2* q = reinterpret_cast<float2*>(out + i * K.plane + g);
                    if constexpr (AVG)
                        v = fma(V2(wp), V2(*reinterpret_cast<const float2*>(pv + i * K.plane + g)),
                                V2(wn) * v);
                    *q = v.v;
                } else if (act0) {
                    float* q = out + i * K.plane + g;
                    *q = AVG ? fmaf(wp, pv[i * K.plane + g], wn * v.x()) : v.x();
                }
            };
#define PX(i) nnd_pos_x(load6(plane_row(ring, (i), y), lx))
#define NX(i) nnd_neg_x(load6(plane_row(ring, (i), y), lx))
#define PY(i) nnd_pos_y(ldv(up_m2 + pindex(i) * RW + lx), ldv(up_m1 + pindex(i) * RW + lx), f[i], \
                        ldv(up_p1 + pindex(i) * RW + lx))
#define NY(i) nnd_neg_y(ldv(dn_m1 + pindex(i) * RW + lx), f[i], ldv(dn_p1 + pindex(i) * RW + lx), \
                        ldv(dn_p2 + pindex(i) * RW + lx))
#pragma unroll
            for (int o = 0; o < 2; o++) { // axis orbits 0, 2
                const int i0 = 8 * o;
                const float cxs = K.c[2 * o] * K.inv_dx, cys = K.c[2 * o] * K.inv_dy;
                put(i0 + 0, cxs * PX(i0 + 0));
                put(i0 + 1, cys * PY(i0 + 1));
                put(i0 + 2, -cxs * NX(i0 + 2));
                put(i0 + 3, -cys * NY(i0 + 3));
            }
#pragma unroll
            for (int o = 0; o < 2; o++) { // diagonal orbits 1, 3
                const int i0 = 4 + 8 * o;
                const float cxs = K.c[2 * o + 1] * K.inv_dx, cys = K.c[2 * o + 1] * K.inv_dy;
                put(i0 + 0, fma(cxs, PX(i0 + 0), cys * PY(i0 + 0)));
                put(i0 + 1, fma(cys, PY(i0 + 1), -cxs * NX(i0 + 1)));
                put(i0 + 2, -(fma(cxs, NX(i0 + 2), cys * NY(i0 + 2))));
                put(i0 + 3, fma(cxs, PX(i0 + 3), -cys * NY(i0 + 3)));
            }
#undef PX
#undef NX
#undef PY
#undef NY
            if (act1) {
                float2* q = reinterpret_cast<float2*>(out + 16 * K.plane + g);
                if constexpr (AVG)
                    ln = fma(V2(wp), V2(*reinterpret_cast<const float2*>(pv + 16 * K.plane + g)),
                             V2(wn) * ln);
                *q = ln.v;
            } else if (act0) {
                float* q = out + 16 * K.plane + g;
                *q = AVG ? fmaf(wp, pv[16 * K.plane + g], wn * ln.x()) : ln.x();
            }

            // TNE statistics of the state being stepped (Eqs. (90)-(91)); sums of Delta_k
            // and d^2 accumulate as packed pairs, folded at the end of the strip
            if (do_tne) {
                if (act1) {
                    V2 d2(0.f);
#pragma unroll
                    for (int k = 0; k < TNE_K; k++) {
                        const V2 Dk = D[k];
                        d2 = fma(Dk, Dk, d2);
                        tsp[k] += Dk;
                        tsm[TNE_K + k] += fabsf(Dk.x()) + fabsf(Dk.y());
                        tmin[k] = fminf(tmin[k], fminf(Dk.x(), Dk.y()));
                        tmax[k] = fmaxf(tmax[k], fmaxf(Dk.x(), Dk.y()));
                    }
                    tsm[2 * TNE_K] += sqrt_approx(d2.x()) + sqrt_approx(d2.y());
                    td2 += d2;
                } else if (act0) {
                    float d2 = 0.f;
#pragma unroll
                    for (int k = 0; k < TNE_K; k++) {
                        const float Dk = D[k].x();
                        d2 = fmaf(Dk, Dk, d2);
                        tsp[k] += V2(Dk, 0.f);
                        tsm[TNE_K + k] += fabsf(Dk);
                        tmin[k] = fminf(tmin[k], Dk);
                        tmax[k] = fmaxf(tmax[k], Dk);
                    }
                    tsm[2 * TNE_K] += sqrt_approx(d2);
                    td2 += V2(d2, 0.f);
                }
            }
        }
        cp_wait<0>();
        if (do_tne) { // per strip: warp sums in FP32, then FP64 per warp
#pragma unroll
            for (int k = 0; k < TNE_K; k++) tsm[k] = tsp[k].x() + tsp[k].y();
            tsm[2 * TNE_K + 1] = td2.x() + td2.y();
#pragma unroll
            for (int q = 0; q < NSUM; q++) {
                const float v = warp_sum(tsm[q]);
                if (lane == 0) tsum[warp * NSUM + q] += (double)v;
            }
        }
    }

    // end of step: status, TNE partials, arrival count; the last block finishes
    if (__syncthreads_or(bad) && tid == 0) atomicOr(&a.ctr->status, 1);
    if (do_tne) {
#pragma unroll
        for (int k = 0; k < TNE_K; k++) {
            const float mn = warp_min(tmin[k]), mx = warp_max(tmax[k]);
            if (lane == 0) {
                tmm[warp * NMM + k] = mn;
                tmm[warp * NMM + TNE_K + k] = mx;
            }
        }
        __syncthreads();
        double* part = a.partials + blockIdx.x; // quantity-major, stride gridDim.x
        const size_t ps = gridDim.x;
        for (int q = tid; q < NSUM; q += MT) {
            double sacc = 0.0;
            for (int w = 0; w < NWM; w++) sacc += tsum[w * NSUM + q];
            part[ps * (q < 2 * TNE_K ? q : 4 * TNE_K + (q - 2 * TNE_K))] = sacc;
        }
        for (int q = tid; q < NMM; q += MT) {
            float v = tmm[q];
            for (int w = 1; w < NWM; w++)
                v = q < TNE_K ? fminf(v, tmm[w * NMM + q]) : fmaxf(v, tmm[w * NMM + q]);
            part[ps * (2 * TNE_K + q)] = (double)v;
        }
        __threadfence();
    }
    __syncthreads();
    __shared__ unsigned int s_last;
    if (tid == 0) s_last = (atomicAdd(&a.ctr->arrivals, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last && tid == 0) { // the grid-wide TNE record is finished by launch_tne_finish
        if (do_tne) {
            a.ctr->hist_count += 1;
            a.ctr->tne_step = step;
        }
        if (a.stage < 2) a.ctr->tne_pending = do_tne ? 1 : 0;
        if (a.stage == 0 || a.stage == 2) a.ctr->step = step + 1;
        a.ctr->arrivals = 0u;
    }
}

template <int REC, bool GEN, bool AVG>
cudaError_t march_prepare()
{
    static cudaError_t done = cudaFuncSetAttribute(march_kernel<REC, GEN, AVG>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)MARCH_SMEM);
    return done;
}

// resident blocks per SM of a variant; the averaging stage of a step shares the grid
// of its first stage, so both must fit that many blocks (checked at launch)
template <int REC, bool GEN, bool AVG>
int resident_of()
{
    static int per_sm = -1;
    if (per_sm < 0) {
        if (march_prepare<REC, GEN, AVG>() != cudaSuccess) return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_kernel<REC, GEN, AVG>,
                                                          MT, MARCH_SMEM) != cudaSuccess)
            return -1;
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

template <int REC, bool GEN>
int resident_min()
{
    const int a = resident_of<REC, GEN, false>(), b = resident_of<REC, GEN, true>();
    return a < 0 || b < 0 ? -1 : (a < b ? a : b);
}

} // namespace

// Blocks resident on the whole GPU, and the strip height: the number of strips
// per column of the grid is chosen so that the strips fill whole waves of the
// resident blocks while each strip stays long compared with its 3-row
// prologue (rows staged and macros recovered before the first update).
// mode = recovery | (general boundaries << 1): the general variant carries walls,
// Dirichlet and specular sides; the plain one only index maps.
namespace {
int resident_blocks(int mode)
{
    static int sms = -1;
    if (sms < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int m = mode & 3;
    const int per_sm = m == 0 ? resident_min<0, false>()
                       : m == 1 ? resident_min<1, false>()
                       : m == 2 ? resident_min<0, true>() : resident_min<1, true>();
    return per_sm < 0 ? -1 : per_sm * sms;
}
} // namespace

void march_plan(int mode, int nx, int ny, int* grid, int* strip_rows)
{
    const int G = resident_blocks(mode);
    const int nsx = (nx + BW - 1) / BW;
    // 32-row strips measured best at 4096^2 (16: -12 %, 64: -11 %, one wave of
    // 293-row strips: -36 %); smaller grids use shorter strips so that every
    // resident block gets work
    int rows = 32;
    while (rows > 8 && (long)nsx * ((ny + rows - 1) / rows) < G) rows /= 2;
    if (rows > ny) rows = ny;
    if (const char* env = getenv("LBKM_MARCH_ROWS")) { // tuning override
        const int r = atoi(env);
        if (r >= 1) rows = r < ny ? r : ny;
    }
    const long strips = (long)nsx * ((ny + rows - 1) / rows);
    *grid = G < 0 ? -1 : (int)(strips < G ? strips : G);
    *strip_rows = rows;
}

int march_grid(int mode, int nx, int ny)
{
    int g, r;
    march_plan(mode, nx, ny, &g, &r);
    return g;
}

namespace {
template <int REC, bool GEN>
void launch_variant(bool avg, const ModelConst<float>& K, const StepLaunch& a, int rows,
                    cudaStream_t s)
{
    if (avg)
        march_kernel<REC, GEN, true><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows);
    else
        march_kernel<REC, GEN, false><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows);
}
} // namespace

cudaError_t launch_march(int mode, const ModelConst<float>& K, const StepLaunch& a, cudaStream_t s)
{
    int g, rows;
    march_plan(mode, K.nx, K.ny, &g, &rows);
    if (g < 0) return cudaErrorInvalidConfiguration;
    if (g != a.grid) return cudaErrorInvalidConfiguration; // partial buffers sized for a.grid
    const bool avg = a.stage >= 2;
    switch (mode & 3) {
    case 0: launch_variant<0, false>(avg, K, a, rows, s); break;
    case 1: launch_variant<1, false>(avg, K, a, rows, s); break;
    case 2: launch_variant<0, true>(avg, K, a, rows, s); break;
    default: launch_variant<1, true>(avg, K, a, rows, s); break;
    }
    return cudaGetLastError();
}

} // namespace lbk
