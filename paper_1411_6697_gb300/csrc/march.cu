// march.cu -- the FP32 2-D step kernel: y-marching strips, two rows per iteration,
// two cells per thread, rows moved by bulk asynchronous copies in both directions.
//
// A block of 128 threads (4 warps) owns a strip of 128 columns x `strip_rows` rows
// and marches up it two rows per iteration: warps 0-1 (warp pair 0) update row y,
// warps 2-3 (warp pair 1) row y + 1. Thread t of a warp pair updates the cells
// (x0 + 2t, y + r) and (x0 + 2t + 1, y + r) together, so most arithmetic runs as
// packed FP32 pairs. Two blocks share an SM.
//
// Shared memory holds a ring of eight staged rows (row r in slot r & 7), each with
// all 17 planes: rows y-2..y+3 are read in an iteration (stencils, and the recovery
// of rows y+2, y+3), rows y+4, y+5 are in flight. Each staged plane row holds columns
// x0-4 .. x0+131 and is filled by one bulk asynchronous copy (the TMA unit's
// non-tensor mode: both addresses and the size multiples of 16 bytes) completing on
// an mbarrier per pair of rows; columns no such copy can reach (the wrapped or clamped
// halo at the grid's x-edges, the tail of a row whose length is not a multiple of 4,
// ghost rows of Dirichlet or specular sides) are filled by per-element asynchronous
// copies that arrive on the same mbarrier, or by stores of the side's equilibrium.
// The updated rows are written into an output buffer in shared memory and leave by
// bulk asynchronous stores (the few columns of a row tail past its last multiple of 4
// by plain stores).
//
// Per iteration (rows y, y+1): wait for rows y+2, y+3; warp pair r recovers rho, u, T
// of row y+2+r from its exact conserved sums (kept in registers: the same pair
// updates that row in the next iteration; u, v also go to a ring of eight rows for
// the neighbours' gradients); one barrier; warp pair r updates row y+r into the
// output buffer; one barrier; warp 0 and warps 2-3 issue the copies of rows y+6, y+7
// into the slots of rows y-2, y-1, warp 1 the stores of rows y, y+1.
// The conserved moments are summed exactly (double-float butterflies); rho, u, T are
// then formed in FP64 (REC = 0) or in double-float on the FP32 pipes (REC = 1), and
// the ignition test T > T_ig is taken in that precision. The TNE statistics of the
// updated state's input (Delta_5..Delta_16, Sec. VI, Eqs. (90)-(91)) accumulate per
// thread over a strip (32 cells per column), the sums of Delta_k and |Delta_k| exactly
// (TwoSum pairs), and from there on in FP64.
#include <cuda.h>
#include <float.h>
#include <stdlib.h>

#include "cell.cuh"
#include "kernels.cuh"
#include "pair.cuh"
#include "reduce.cuh"
#include "vec2.cuh"

namespace lbk {

namespace {

constexpr int MT = 128;          // threads per block
constexpr int NWM = MT / 32;     // warps per block
constexpr int BW = 128;          // columns per strip
constexpr int XO = 4;            // column x0 sits at element XO of a staged row
constexpr int RW = BW + 2 * XO;  // staged row: columns x0-4 .. x0+BW+3 (544 bytes)
constexpr int NSLOT = 8;         // staged rows kept: y-2 .. y+5, in four row pairs
constexpr int PST = 2 * RW;      // floats from one plane of a row pair to the next
// a row pair's slot: [plane][row of the pair][RW], as a tensor copy of a box of RW
// columns x 2 rows x 17 planes lays it out, padded to a multiple of 128 bytes (the
// alignment of a tensor copy's shared-memory address)
constexpr int PSLOT = (NPLANE * PST * 4 + 127) / 128 * 128 / 4;

// shared-memory layout (floats from a 128-byte aligned start)
constexpr int OBUF = NSLOT / 2 * PSLOT;          // updated rows: [NPLANE][2][BW]
constexpr int UVB = OBUF + NPLANE * 2 * BW;      // (u, v) of rows: [NSLOT][2][RW]
constexpr int SMEM_FLOATS = UVB + NSLOT * 2 * RW;
static_assert(RW % 4 == 0 && PSLOT % 32 == 0 && OBUF % 32 == 0 && UVB % 4 == 0,
              "staged rows on 16-byte, row-pair slots and the output rows on 128-byte boundaries");
constexpr size_t OFF_TSUM = (size_t)SMEM_FLOATS * 4;            // double[NSUM]
constexpr size_t OFF_TMM = OFF_TSUM + (size_t)NSUM * 8;           // float[NWM][NMM]
constexpr size_t OFF_MBAR = (OFF_TMM + (size_t)NWM * NMM * 4 + 15) / 16 * 16;
constexpr int NMB = 4;                                            // row pairs in flight or in use
constexpr size_t MARCH_SMEM = OFF_MBAR + NMB * 8 + 128;           // + room to align the start
static_assert(MARCH_SMEM <= 112 * 1024, "two blocks per SM need <= 112 KB each");
static_assert(2 * NSUM * MT <= OBUF && 4 * NSUM <= MT,
              "the strip's TNE partials fit in the idle ring, four threads per sum");
constexpr uint32_t PAIR_BYTES = NPLANE * PST * 4; // one tensor copy of a row pair

// staged row r (plane p at + p * PST) and plane p of it
__device__ __forceinline__ float* srow(float* ring, int r)
{
    return ring + ((r >> 1) & (NSLOT / 2 - 1)) * PSLOT + (r & 1) * RW;
}
__device__ __forceinline__ float* plane_row(float* ring, int p, int r) { return srow(ring, r) + p * PST; }
__device__ __forceinline__ float* uv_row(float* smem_f, int r, int field)
{
    return smem_f + UVB + ((r & (NSLOT - 1)) * 2 + field) * RW;
}

// ---------------- mbarriers and bulk copies -------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
}
// one bounded wait for the phase with the given parity; false if it did not complete
__device__ __forceinline__ bool mbar_try(uint32_t mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
// waits with a bound (about 20 ms of suspended polling); false if the bound ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity)
{
    for (int i = 0; i < 20000; i++)
        if (mbar_try(mb, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mb)
        : "memory");
}
// a box of RW columns x 2 rows x 17 planes from column x, row y (tensor map of the input)
__device__ __forceinline__ void tma_load_pair(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t mb)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(tm), "r"(x), "r"(y), "r"(0), "r"(mb)
        : "memory");
}
// a box of BW columns x 2 rows x 17 planes to column x, row y (tensor map of the output;
// parts of the box outside the grid are not written)
__device__ __forceinline__ void tma_store_pair(const CUtensorMap* tm, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tm),
                 "r"(x), "r"(y), "r"(0), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_arrive_noinc(uint32_t mb)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
}
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Where plane p of staged row r comes from: the grid row gy and plane sp (specular
// sides mirror the row and reverse v_y), or a Dirichlet side (dir >= 0) whose
// equilibrium fills the row.
template <bool GEN>
__device__ __forceinline__ void row_source(const ModelConst<float>& K, int r, int p, int& gy, int& sp,
                                           int& dir)
{
    gy = r;
    sp = p;
    dir = -1;
    if (r >= 0 && r < K.ny) return;
    if constexpr (!GEN) {
        gy = map_index(r, K.ny, K.bc_y);
    } else {
        const int s = r < 0 ? 2 : 3, code = K.sbc[s];
        if (code == 3) {
            dir = s;
        } else if (code == 4) {
            gy = r < 0 ? -r - 1 : 2 * K.ny - 1 - r;
            gy = gy < 0 ? 0 : (gy >= K.ny ? K.ny - 1 : gy);
            sp = mirror_plane(p);
        } else {
            gy = map_index(r, K.ny, code == 0 ? 0 : 1);
        }
    }
}

// Issue the copies of staged rows ra, ra+1 (pair mbarrier mb) for the strip at x0;
// rows above rmax are not needed. A pair whose rows and staged columns all lie inside
// the grid arrives by one tensor copy (thread 0). Otherwise warp 0: one bulk copy per
// plane row for the columns
// [cs, ce) (16-byte aligned), after arming the mbarrier with their byte count.
// Warps 2-3: the remaining columns x0-2 .. x0+BW+1 that active cells read (edges of
// the grid, a row tail past the last multiple of 4, Dirichlet rows), element by
// element, then one arrival each on the mbarrier once their copies have landed.
template <bool GEN>
__device__ __forceinline__ void issue_pair(const float* __restrict__ in, float* ring, uint32_t mb,
                                           int ra, int rmax, int x0, const ModelConst<float>& K,
                                           const CUtensorMap* tm)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // both rows inside the grid, every staged column inside it: one tensor copy
    if (x0 >= XO && x0 + BW + XO <= K.nx && ra >= 0 && ra + 1 < K.ny) {
        if (tid == 0) {
            mbar_expect_tx(mb, PAIR_BYTES);
            fence_async_shared();
            tma_load_pair(smem_addr(srow(ring, ra)), tm, x0 - XO, ra, mb);
        } else if (warp >= 2) {
            cp_arrive_noinc(mb);
        }
        return;
    }
    const int nx4 = K.nx & ~3;
    const int cs = x0 - XO > 0 ? x0 - XO : 0;
    const int ce = x0 + BW + XO < nx4 ? x0 + BW + XO : nx4;
    if (warp == 0) {
        const float* src[2];
        uint32_t dst[2], nb[2];
        uint32_t bytes = 0;
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int task = lane + 32 * u;
            nb[u] = 0;
            if (task < 2 * NPLANE) {
                const int r = ra + task / NPLANE, p = task % NPLANE;
                int gy, sp, dir;
                row_source<GEN>(K, r, p, gy, sp, dir);
                if (r <= rmax && dir < 0 && ce > cs) {
                    src[u] = in + sp * K.plane + (int64_t)gy * K.pitch + cs;
                    dst[u] = smem_addr(plane_row(ring, p, r) + (cs - (x0 - XO)));
                    nb[u] = (uint32_t)(ce - cs) * 4u;
                    bytes += nb[u];
                }
            }
        }
        bytes = __reduce_add_sync(0xffffffffu, bytes);
        if (lane == 0) mbar_expect_tx(mb, bytes);
        __syncwarp();
        fence_async_shared();
#pragma unroll
        for (int u = 0; u < 2; u++)
            if (nb[u]) bulk_g2s(dst[u], src[u], nb[u], mb);
    } else if (warp >= 2) {
        // nothing to fill when the bulk copies cover columns x0-2 .. x0+BW+1 and no row
        // of the pair is a Dirichlet ghost row
        bool need = x0 - 2 < cs || ce < x0 + BW + 2;
        if constexpr (GEN)
            need = need || (ra < 0 && K.sbc[2] == 3) || (ra + 1 >= K.ny && ra + 1 <= rmax && K.sbc[3] == 3);
        if (!need) {
            cp_arrive_noinc(mb);
            return;
        }
        const int ft = tid - 64; // 0..63
        // tasks: (row, plane, side) with side 0 = columns [x0-2, cs), side 1 = columns
        // [max(ce, x0-2), min(nx+4, x0+BW+2)) (the ghost columns active cells read, and
        // two more that only an inactive neighbour reads; with periodic or zero-gradient
        // sides every column up to x0+BW+2, so that a cell past the grid holds a real
        // cell's values); Dirichlet rows: every column
        for (int task = ft; task < 4 * NPLANE; task += 64) {
            const int side = task & 1, rp = task >> 1;
            const int r = ra + rp / NPLANE, p = rp % NPLANE;
            if (r > rmax) continue;
            int gy, sp, dir;
            row_source<GEN>(K, r, p, gy, sp, dir);
            float* row = plane_row(ring, p, r);
            int c0, c1;
            if (dir >= 0) { // the whole row holds the side's equilibrium (split between sides)
                c0 = side ? x0 + BW / 2 : x0 - 2;
                c1 = side ? x0 + BW + 2 : x0 + BW / 2;
            } else {
                c0 = side ? (ce > x0 - 2 ? ce : x0 - 2) : x0 - 2;
                c1 = side ? (!GEN ? x0 + BW + 2 : (K.nx + 4 < x0 + BW + 2 ? K.nx + 4 : x0 + BW + 2)) : cs;
                if (!side && ce <= cs) c1 = x0 - 2; // no bulk copy: side 1 takes the row
                if (side && ce <= cs) c0 = x0 - 2;
            }
            for (int x = c0; x < c1; x++) {
                float* d = row + (x - (x0 - XO));
                if (dir >= 0) {
                    *d = K.sfeq[dir][p];
                    continue;
                }
                int xx = x, psrc = sp;
                if (x < 0 || x >= K.nx) {
                    const int s = x < 0 ? 0 : 1;
                    if constexpr (GEN) {
                        if (K.sbc[s] == 3) {
                            *d = K.sfeq[s][p];
                            continue;
                        }
                        xx = map_index(x, K.nx, K.sbc[s] == 0 ? 0 : 1);
                    } else {
                        xx = map_index(x, K.nx, K.bc_x);
                    }
                }
                cp4(smem_addr(d), in + psrc * K.plane + (int64_t)gy * K.pitch + xx);
            }
        }
        cp_arrive_noinc(mb);
    }
}

// Walls (Sec. IV.D): a staged ghost row r_ghost holds a copy of the fluid row r_src (the
// index map clamps); add the non-equilibrium-extrapolation correction to the thread's
// own two columns of its 16 f planes (lambda stays a copy).
__device__ __forceinline__ void wall_fix_row(float* ring, int r_ghost, int r_src, int side,
                                             const ModelConst<float>& K, int lx)
{
    V2 f[16], d[16];
#pragma unroll
    for (int i = 0; i < 16; i++) f[i] = ldv(plane_row(ring, i, r_src) + lx);
    wall_correction(K, f, side, d);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        float* q = plane_row(ring, i, r_ghost) + lx;
        *reinterpret_cast<float2*>(q) = (ldv(q) + d[i]).v;
    }
}
// wall correction of staged row r if it is a wall ghost row
template <bool GEN>
__device__ __forceinline__ void wall_fix(float* ring, int r, const ModelConst<float>& K, int lx)
{
    if constexpr (GEN) {
        if (r < 0 && K.sbc[2] == 2) wall_fix_row(ring, r, 0, 0, K, lx);
        if (r >= K.ny && K.sbc[3] == 2) wall_fix_row(ring, r, K.ny - 1, 1, K, lx);
    }
}

struct Mac {
    V2 rho, ux, uy, T;
    bool ig0, ig1;
};

// rho, u, T of the thread's two cells of staged row r (exact conserved sums, then FP64
// or double-float); u, v also into the (u, v) ring, with the halo columns x0-1 and
// x0+BW (plain FP32 velocity, used only in grad u) by the first and last thread.
template <int REC>
__device__ __forceinline__ Mac recover_row(float* smem_f, float* ring, int r, int t,
                                           const ModelConst<float>& K, const DfConst& C, int& bad,
                                           bool act0, bool act1)
{
    const int lx = XO + 2 * t;
    V2 f[16];
#pragma unroll
    for (int i = 0; i < 16; i++) f[i] = ldv(plane_row(ring, i, r) + lx);
    Mac o;
    bool ok0, ok1;
    recover_pair_fast<REC>(f, C, K, o.rho, o.ux, o.uy, o.T, o.ig0, o.ig1, ok0, ok1);
    if ((act0 && !ok0) || (act1 && !ok1)) bad = 1;
    float* ur = uv_row(smem_f, r, 0);
    float* vr = uv_row(smem_f, r, 1);
    *reinterpret_cast<float2*>(ur + lx) = o.ux.v;
    *reinterpret_cast<float2*>(vr + lx) = o.uy.v;
    if (t == 0 || t == 63) {
        const int hx = t == 0 ? XO - 1 : XO + BW;
        float g[16], hu, hv;
#pragma unroll
        for (int i = 0; i < 16; i++) g[i] = plane_row(ring, i, r)[hx];
        velocity_f32(g, K, hu, hv);
        ur[hx] = hu;
        vr[hx] = hv;
    }
    return o;
}

// per-thread TNE statistics of one strip and of the whole launch (min, max). The sums of
// Delta_k and |Delta_k| are carried as unevaluated pairs s + c of FP32 values: every
// addition's rounding error is recovered exactly (TwoSum) and added to c, so s + c is the
// exact sum of the FP32 terms up to the rounding of c itself (of order u^2 per term,
// u = 2^-24). The sums of d and d^2 (one-signed, each term already rounded to about 12 u
// by its own FP32 evaluation) are plain FP32 sums of at most 32 terms per column
// (relative error <= 31 u). Past the thread everything is FP64.
struct TneAcc {
    V2 sum[TNE_K], abs[TNE_K], dsum, d2sum; // the two cells of the thread apart
    float sumc[TNE_K], absc[TNE_K];         // the compensating terms, both columns
};

__device__ __forceinline__ void acc_exact(V2& s, float& c, V2 x)
{
    const D2 t = two_sum(s, x);
    s = t.hi;
    c += t.lo.x() + t.lo.y();
}

// ---------------- the update of one row by one warp pair -------------------------
// Row y, the thread's cells x0 + 2t and x0 + 2t + 1 (active when act0 / act1), macros
// mc recovered in the previous iteration; the results go to the output rows ob
// (17 planes of BW floats). TNE: the row's TNE statistics join the thread's sums. With
// periodic or zero-gradient sides (!GEN) a cell past the grid's last column holds a real
// cell's values (staging fills the whole box through the side map), so the statistics
// run without a branch: the sums take Delta_k times the lane mask am (1 active, 0 not),
// the extremes the unmasked values. With general sides they take the active cells only.
template <int REC, bool AVG, bool SRT, bool TNE, bool GEN>
__device__ __forceinline__ void update_row(float* smem_f, float* ring, float* ob, int y, int x0,
                                           int t, const ModelConst<float>& K, const StepLaunch& a,
                                           const Mac& mc, bool act0, bool act1, V2 am, TneAcc& acc,
                                           float* tmin, float* tmax)
{
    const int lx = XO + 2 * t;
    const float dt = K.dt;
    const V2 rho = mc.rho, ux = mc.ux, uy = mc.uy, T = mc.T;
    float* r0 = srow(ring, y);

    // reaction over dt (Eq. (28)), decided by the recovered T
    const V2 rT = rho * T;
    const float* lm = r0 + 16 * PST;
    const V2 lam0 = ldv(lm + lx);
    const float ri0 = reaction_increment(lam0.x(), K.omega1 * rT.x(), K.omega2 * rT.x(), dt);
    const float ri1 = reaction_increment(lam0.y(), K.omega1 * rT.y(), K.omega2 * rT.y(), dt);
    const V2 dlam(mc.ig0 ? ri0 : 0.f, mc.ig1 ? ri1 : 0.f);
    const V2 cr = dlam * K.chem;

    V2 W[16]; // M^-1 of the moment-space collision, or of S f_hat^eq + C_hat (SRT)
    if constexpr (SRT) {
        // single-relaxation-time collision (Sec. V, Eq. (87)): Omega = -S (f - f^eq) + C
        // with f^eq = M^-1 f_hat^eq and C = M^-1 C_hat, i.e. W - S f with
        // W = M^-1 (S f_hat^eq + C_hat); the rates being equal, A_hat vanishes
        // (Eqs. (3)-(4)) and no forward transform is needed
        const float Srt = K.S[4];
        V2 q[16], dq[16];
        feq_moments(V2(K.DI), rho, ux, uy, T, q);
        dfeq_dT(V2(K.DI), rho, ux, uy, T, dq);
#pragma unroll
        for (int k = 0; k < 16; k++) q[k] = k < 3 ? V2(Srt) * q[k] : fma(V2(Srt), q[k], dq[k] * cr);
        inverse_moments(K, q, W);
    } else {
    // moments, equilibrium, non-equilibrium parts (Delta_1..4 vanish)
    V2 m[16];
    {
        V2 f[16];
#pragma unroll
        for (int i = 0; i < 16; i++) f[i] = ldv(r0 + i * PST + lx);
        forward_moments(K, f, m);
    }
    {
        V2 q[16];
        feq_moments(V2(K.DI), rho, ux, uy, T, q);
#pragma unroll
        for (int k = 4; k < 16; k++) m[k] = m[k] - q[k];
    }
    // TNE statistics of the state being stepped (Eqs. (90)-(91)); a cell past the grid's
    // last column contributes nothing
    if constexpr (TNE) {
        auto both = [&](V2 mask) {
            V2 d2(0.f);
#pragma unroll
            for (int k = 0; k < TNE_K; k++) {
                const V2 Dk = m[k + 4], Dm = Dk * mask;
                d2 = fma(Dm, Dm, d2);
                acc_exact(acc.sum[k], acc.sumc[k], Dm);
                acc_exact(acc.abs[k], acc.absc[k], V2(fabsf(Dm.x()), fabsf(Dm.y())));
                tmin[k] = fmin3(tmin[k], Dk.x(), Dk.y());
                tmax[k] = fmax3(tmax[k], Dk.x(), Dk.y());
            }
            acc.dsum += V2(sqrt_approx(d2.x()), sqrt_approx(d2.y()));
            acc.d2sum += d2;
        };
        if constexpr (!GEN) {
            both(am);
        } else if (act1) {
            both(V2(1.f));
        } else if (act0) { // the last cell of a row, alone in its pair
            float d2 = 0.f;
#pragma unroll
            for (int k = 0; k < TNE_K; k++) {
                const float Dk = m[k + 4].x();
                d2 = fmaf(Dk, Dk, d2);
                acc_exact(acc.sum[k], acc.sumc[k], V2(Dk, 0.f));
                acc_exact(acc.abs[k], acc.absc[k], V2(fabsf(Dk), 0.f));
                tmin[k] = fminf(tmin[k], Dk);
                tmax[k] = fmaxf(tmax[k], Dk);
            }
            acc.dsum += V2(sqrt_approx(d2), 0.f);
            acc.d2sum += V2(d2, 0.f);
        }
    }

    // grad u: x from the (u, v) row y (halo columns included), y from rows y+-1
    const float* uxr = uv_row(smem_f, y, 0);
    const float* uyr = uv_row(smem_f, y, 1);
    const float2 uxl = *reinterpret_cast<const float2*>(uxr + lx - 2);
    const float2 uxh = *reinterpret_cast<const float2*>(uxr + lx + 2);
    const float2 uyl = *reinterpret_cast<const float2*>(uyr + lx - 2);
    const float2 uyh = *reinterpret_cast<const float2*>(uyr + lx + 2);
    const V2 dux_dx = (V2(ux.y(), uxh.x) - V2(uxl.y, ux.x())) * K.half_inv_dx;
    const V2 duy_dx = (V2(uy.y(), uyh.x) - V2(uyl.y, uy.x())) * K.half_inv_dx;
    const V2 dux_dy = (ldv(uv_row(smem_f, y + 1, 0) + lx) - ldv(uv_row(smem_f, y - 1, 0) + lx)) *
                      K.half_inv_dy;
    const V2 duy_dy = (ldv(uv_row(smem_f, y + 1, 1) + lx) - ldv(uv_row(smem_f, y - 1, 1) + lx)) *
                      K.half_inv_dy;
    const V2 theta = (dux_dx + duy_dy) * K.inv_DI;
    const V2 shear = duy_dx + dux_dy;
    const V2 A8 = (rT * K.A8c) * fma(V2(4.f) * ux, dux_dx - theta, V2(2.f) * uy * shear);
    const V2 A9 = (rT * K.A9c) * fma(V2(4.f) * uy, duy_dy - theta, V2(2.f) * ux * shear);

    // collision in moment space and back
    {
        V2 dq[16], Om[16];
        dfeq_dT(V2(K.DI), rho, ux, uy, T, dq);
        Om[0] = Om[1] = Om[2] = V2(0.f);
        Om[3] = dq[3] * cr;
#pragma unroll
        for (int k = 4; k < 16; k++) Om[k] = fma(V2(-K.S[k]), m[k], dq[k] * cr);
        Om[7] += A8;
        Om[8] += A9;
        inverse_moments(K, Om, W);
    }

    }

    // results into the output rows; a later SSP Runge-Kutta stage (AVG) writes
    // wp * u^n + wn * E(in), u^n read from prev at the cell's own position
    const int64_t g = (int64_t)y * K.pitch + x0 + 2 * t;
    const float* pv = static_cast<const float*>(a.prev);
    const float wp = (float)a.wprev, wn = (float)a.wnew;
    auto store = [&](int i, V2 v) {
        if constexpr (AVG) {
            if (act1)
                v = fma(V2(wp), V2(*reinterpret_cast<const float2*>(pv + i * K.plane + g)), V2(wn) * v);
            else if (act0)
                v = V2(fmaf(wp, pv[i * K.plane + g], wn * v.x()), 0.f);
        }
        *reinterpret_cast<float2*>(ob + i * 2 * BW + 2 * t) = v.v;
    };

    // lambda: u . grad(lambda) with NND interface values
    const float* rm2 = srow(ring, y - 2);
    const float* rm1 = srow(ring, y - 1);
    const float* rp1 = srow(ring, y + 1);
    const float* rp2 = srow(ring, y + 2);
    {
        const Q6 lq = load6(lm, lx);
        const V2 lpx = nnd_pos_x(lq), lnx = nnd_neg_x(lq);
        const V2 lm1 = ldv(rm1 + 16 * PST + lx);
        const V2 lp1 = ldv(rp1 + 16 * PST + lx);
        const V2 lpy = nnd_pos_y(ldv(rm2 + 16 * PST + lx), lm1, lam0, lp1);
        const V2 lny = nnd_neg_y(lm1, lam0, lp1, ldv(rp2 + 16 * PST + lx));
        const V2 lax(ux.x() > 0.f ? lpx.x() : lnx.x(), ux.y() > 0.f ? lpx.y() : lnx.y());
        const V2 lay(uy.x() > 0.f ? lpy.x() : lny.x(), uy.y() > 0.f ? lpy.y() : lny.y());
        const V2 ladv = fma(ux * K.inv_dx, lax, uy * K.inv_dy * lay);
        V2 ln = fma(V2(-dt), ladv, lam0) + dlam;
        ln = vmin(vmax(ln, V2(0.f)), V2(1.f));
        store(16, ln);
    }

    // NND flux differences (upwind side fixed per velocity), Euler update
    auto put = [&](int i, V2 f0, V2 adv) {
        V2 w = W[i];
        if constexpr (SRT) w = fma(V2(-K.S[4]), f0, w); // the -S f of the SRT collision
        store(i, fma(V2(dt), w - adv, f0));
    };
#define F0(i) ldv(r0 + (i) * PST + lx)
#define PX(i) nnd_pos_x(load6(r0 + (i) * PST, lx))
#define NX(i) nnd_neg_x(load6(r0 + (i) * PST, lx))
#define PY(i, f0) nnd_pos_y(ldv(rm2 + (i) * PST + lx), ldv(rm1 + (i) * PST + lx), f0, ldv(rp1 + (i) * PST + lx))
#define NY(i, f0) nnd_neg_y(ldv(rm1 + (i) * PST + lx), f0, ldv(rp1 + (i) * PST + lx), ldv(rp2 + (i) * PST + lx))
#pragma unroll
    for (int o = 0; o < 2; o++) { // axis orbits 0, 2
        const int i0 = 8 * o;
        const float cxs = K.c[2 * o] * K.inv_dx, cys = K.c[2 * o] * K.inv_dy;
        V2 f0;
        f0 = F0(i0 + 0);
        put(i0 + 0, f0, cxs * PX(i0 + 0));
        f0 = F0(i0 + 1);
        put(i0 + 1, f0, cys * PY(i0 + 1, f0));
        f0 = F0(i0 + 2);
        put(i0 + 2, f0, -cxs * NX(i0 + 2));
        f0 = F0(i0 + 3);
        put(i0 + 3, f0, -cys * NY(i0 + 3, f0));
    }
#pragma unroll
    for (int o = 0; o < 2; o++) { // diagonal orbits 1, 3
        const int i0 = 4 + 8 * o;
        const float cxs = K.c[2 * o + 1] * K.inv_dx, cys = K.c[2 * o + 1] * K.inv_dy;
        V2 f0;
        f0 = F0(i0 + 0);
        put(i0 + 0, f0, fma(cxs, PX(i0 + 0), cys * PY(i0 + 0, f0)));
        f0 = F0(i0 + 1);
        put(i0 + 1, f0, fma(cys, PY(i0 + 1, f0), -cxs * NX(i0 + 1)));
        f0 = F0(i0 + 2);
        put(i0 + 2, f0, -(fma(cxs, NX(i0 + 2), cys * NY(i0 + 2, f0))));
        f0 = F0(i0 + 3);
        put(i0 + 3, f0, fma(cxs, PX(i0 + 3), -cys * NY(i0 + 3, f0)));
    }
#undef F0
#undef PX
#undef NX
#undef PY
#undef NY
}

// ---------------- the kernel -----------------------------------------------------
__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// TNE: the TNE statistics are accumulated on every step (the tne_every > 0 handles) and
// reduced into the step's partials when the step is due; no TNE code otherwise
template <int REC, bool GEN, bool AVG, bool SRT, bool TNE>
__global__ void __launch_bounds__(MT, 2)
    march_kernel(const ModelConst<float> K, const StepLaunch a, int strip_rows,
                 const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tensor copies want a 128-byte aligned start
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float* smem_f = reinterpret_cast<float*>(smem);
    float* ring = smem_f;
    float* obuf = smem_f + OBUF;
    double* tsum = reinterpret_cast<double*>(smem + OFF_TSUM);
    float* tmm = reinterpret_cast<float*>(smem + OFF_TMM);
    const uint32_t mbar0 = smem_addr(smem + OFF_MBAR);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wpair = warp >> 1, t = tid & 63, lx = XO + 2 * t;
    const int nx = K.nx, ny = K.ny;
    const float* __restrict__ in = static_cast<const float*>(a.in);
    float* ob = obuf + wpair * BW;

    const DfConst C = df_constants(K);
    const int64_t step = a.ctr->step;
    // AVG stages reduce no TNE
    const bool do_tne = TNE && !AVG && a.tne_every > 0 && (step % a.tne_every) == 0;
    if (tid < NSUM) tsum[tid] = 0.0;
    if (tid < NMB) mbar_init(mbar0 + 8 * tid, 1 + 64);
    fence_async_shared();
    __syncthreads();

    float tmin[TNE_K], tmax[TNE_K];
#pragma unroll
    for (int k = 0; k < TNE_K; k++) tmin[k] = FLT_MAX, tmax[k] = -FLT_MAX;
    int bad = 0;
    bool timeout = false;

    const int nsx = (nx + BW - 1) / BW, nsy = (ny + strip_rows - 1) / strip_rows;
    const int nstrips = nsx * nsy;
    uint32_t q_issued = 0, q_waited = 0; // row pairs of this block, in order
    auto mb_of = [&](uint32_t q) { return mbar0 + 8 * (q % NMB); };
    auto wait_pair = [&](uint32_t q) {
        if (mbar_wait(mb_of(q), (q / NMB) & 1u))
            q_waited = q + 1;
        else
            timeout = true;
    };

    for (int s = blockIdx.x; s < nstrips; s += gridDim.x) {
        const int x0 = (s / nsy) * BW, y0 = (s % nsy) * strip_rows;
        const int yend = y0 + strip_rows < ny ? y0 + strip_rows : ny;
        const int cx = x0 + 2 * t;
        const bool act0 = cx < nx, act1 = cx + 1 < nx;
        const V2 am(act0 ? 1.f : 0.f, act1 ? 1.f : 0.f); // lanes whose cells are in the grid
        const int npairs = (yend - y0 + 5) / 2; // rows y0-2 .. yend+1
        const uint32_t q0 = q_issued;
        TneAcc acc;
#pragma unroll
        for (int k = 0; k < TNE_K; k++) {
            acc.sum[k] = acc.abs[k] = V2(0.f);
            acc.sumc[k] = acc.absc[k] = 0.f;
        }
        acc.dsum = acc.d2sum = V2(0.f);

        __syncthreads(); // the previous strip is done with the ring
        for (int j = 0; j < npairs && j < NMB; j++)
            issue_pair<GEN>(in, ring, mb_of(q0 + j), y0 - 2 + 2 * j, yend + 1, x0, K, &tin);
        q_issued = q0 + (npairs < NMB ? npairs : NMB);
        wait_pair(q0);
        wait_pair(q0 + 1);
        // walls: ghost rows among rows y0-2 .. y0+1 (warp pair 0: y0-1, y0+1; 1: y0-2, y0)
        if constexpr (GEN) {
            wall_fix<GEN>(ring, wpair ? y0 - 2 : y0 - 1, K, lx);
            wall_fix<GEN>(ring, wpair ? y0 : y0 + 1, K, lx);
        }
        __syncthreads();
        // rho, u, T of rows y0 (pair 0) and y0+1 (pair 1), u, v of row y0-1 (pair 0)
        Mac cur = recover_row<REC>(smem_f, ring, y0 + wpair, t, K, C, bad, act0, act1);
        if (wpair == 0) (void)recover_row<REC>(smem_f, ring, y0 - 1, t, K, C, bad, act0, act1);
        if (__syncthreads_or(timeout)) break;

        bool stop = false;
        for (int k = 0;; k++) {
            const int y = y0 + 2 * k;
            if (y >= yend) break;
            if (y + 2 <= yend + 1) wait_pair(q0 + k + 2);
            const int rr = y + 2 + wpair; // the row this pair recovers
            if constexpr (GEN)
                if (rr <= yend + 1) wall_fix<GEN>(ring, rr, K, lx);
            Mac nxt = cur;
            if (rr <= yend) nxt = recover_row<REC>(smem_f, ring, rr, t, K, C, bad, act0, act1);
            if (warp == 1) bulk_wait_read_all(); // the output buffer is free again
            if (__syncthreads_or(timeout)) {
                stop = true;
                break;
            }
            if (y + wpair < yend)
                update_row<REC, AVG, SRT, TNE, GEN>(smem_f, ring, ob, y + wpair, x0, t, K, a, cur,
                                                    act0, act1, am, acc, tmin, tmax);
            cur = nxt;
            fence_async_shared(); // the output rows are read by the bulk stores
            __syncthreads();
            if (warp == 1) {
                // rows y, y+1 leave in one tensor copy; a row at or past ny is clipped (a
                // strip ends on an even row unless it ends at ny)
                if (lane == 0) tma_store_pair(&tout, x0, y, smem_addr(obuf));
            } else if (k + 4 < npairs) {
                issue_pair<GEN>(in, ring, mb_of(q0 + k + 4), y + 6, yend + 1, x0, K, &tin);
            }
            if (k + 4 < npairs) q_issued = q0 + k + 5;
        }
        if (stop) break;
        // the strip's TNE sums: each thread's partials (both columns and the compensating
        // terms) joined in FP64, then added in FP64 in a fixed order: four threads per
        // quantity, 32 partials each, then a shuffle
        if (do_tne) {
            __syncthreads(); // every copy has been waited for: the ring is idle
            double* part = reinterpret_cast<double*>(ring);
            auto join = [](V2 s) { return f2d_fast(s.x()) + f2d_fast(s.y()); };
#pragma unroll
            for (int k = 0; k < TNE_K; k++) {
                part[k * MT + tid] = join(acc.sum[k]) + f2d_fast(acc.sumc[k]);
                part[(TNE_K + k) * MT + tid] = join(acc.abs[k]) + f2d_fast(acc.absc[k]);
            }
            part[2 * TNE_K * MT + tid] = join(acc.dsum);
            part[(2 * TNE_K + 1) * MT + tid] = join(acc.d2sum);
            __syncthreads();
            double s2 = 0.0;
            if (tid < 4 * NSUM) {
                const double* src = part + (tid >> 2) * MT + (tid & 3) * 32;
                double e0 = 0.0, e1 = 0.0;
#pragma unroll 4
                for (int j = 0; j < 32; j += 2) {
                    e0 += src[j];
                    e1 += src[j + 1];
                }
                s2 = e0 + e1;
            }
            s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
            s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
            if (tid < 4 * NSUM && (tid & 3) == 0) tsum[tid >> 2] += s2;
        }
        q_issued = q0 + npairs;
    }
    if (__syncthreads_or(timeout)) {
        // a copy did not land in time: wait (bounded) for every copy still in flight,
        // so none lands after the block has left, and report
        for (uint32_t q = q_waited; q < q_issued; q++) (void)mbar_wait(mb_of(q), (q / NMB) & 1u);
        if (tid == 0) atomicOr(&a.ctr->status, 2);
    }
    if (warp == 1) bulk_wait_all(); // every output row has reached global memory

    // end of step: status, TNE partials, arrival count
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
        for (int q = tid; q < NSUM; q += MT)
            part[ps * (q < 2 * TNE_K ? q : 4 * TNE_K + (q - 2 * TNE_K))] = tsum[q];
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

template <int REC, bool GEN, bool AVG, bool SRT, bool TNE>
cudaError_t march_prepare()
{
    static cudaError_t done = cudaFuncSetAttribute(march_kernel<REC, GEN, AVG, SRT, TNE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)MARCH_SMEM);
    return done;
}

// resident blocks per SM of a variant; the averaging stage of a step shares the grid
// of its first stage, and the single-relaxation-time variant the grid of the general
// one, so all must fit that many blocks (checked at launch)
template <int REC, bool GEN, bool AVG, bool SRT, bool TNE>
int resident_of()
{
    static int per_sm = -1;
    if (per_sm < 0) {
        if (march_prepare<REC, GEN, AVG, SRT, TNE>() != cudaSuccess) return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_kernel<REC, GEN, AVG, SRT, TNE>,
                                                          MT, MARCH_SMEM) != cudaSuccess)
            return -1;
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

template <int REC, bool GEN>
int resident_min()
{
    int r[4] = {resident_of<REC, GEN, false, false, true>(), resident_of<REC, GEN, false, false, false>(),
                resident_of<REC, GEN, true, false, false>(),
                GEN ? 1 << 20 : resident_of<REC, false, false, true, false>()};
    int m = r[0];
    for (int i = 1; i < 4; i++) m = r[i] < 0 || m < 0 ? -1 : (r[i] < m ? r[i] : m);
    return m;
}

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

template <int REC, bool GEN>
void launch_variant(bool avg, bool srt, const ModelConst<float>& K, const StepLaunch& a, int rows,
                    cudaStream_t s)
{
    const CUtensorMap& tin = *reinterpret_cast<const CUtensorMap*>(a.tm_in);
    const CUtensorMap& tout = *reinterpret_cast<const CUtensorMap*>(a.tm_out);
    if (avg)
        march_kernel<REC, GEN, true, false, false><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows, tin, tout);
    else if (srt && !GEN)
        march_kernel<REC, false, false, true, false><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows, tin, tout);
    else if (a.tne_every > 0)
        march_kernel<REC, GEN, false, false, true><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows, tin, tout);
    else
        march_kernel<REC, GEN, false, false, false><<<a.grid, MT, MARCH_SMEM, s>>>(K, a, rows, tin, tout);
}

} // namespace

// Blocks resident on the whole GPU, and the strip height: the number of strips per
// column of the grid is chosen so that the strips fill whole waves of the resident
// blocks while each strip stays long compared with its prologue (four rows staged and
// three recovered before the first update).
// mode = recovery | (general boundaries << 1) | (single relaxation time << 2): the
// general variant carries walls, Dirichlet and specular sides, the plain one only index
// maps; the single-relaxation-time variant exists for the plain forward-Euler step.
void march_plan(int mode, int nx, int ny, int* grid, int* strip_rows)
{
    const int G = resident_blocks(mode);
    const int nsx = (nx + BW - 1) / BW;
    // 64-row strips (4096^2, Gcell/s: 16 rows 14.15, 32 rows 14.97, 48 rows 15.28,
    // 64 rows 15.30, 96 rows 14.61); smaller grids use shorter strips so that every
    // resident block gets work
    int rows = 64;
    while (rows > 8 && (long)nsx * ((ny + rows - 1) / rows) < G) rows /= 2;
    if (rows > ny) rows = ny;
    if (const char* env = getenv("LBKM_MARCH_ROWS")) { // tuning override (even)
        const int r = (atoi(env) + 1) & ~1;
        if (r >= 2) rows = r < ny ? r : ny;
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

// The state viewed as a 3-D tensor (columns, rows, planes) with row stride pitch and
// plane stride plane elements: monotonic strides, 16-byte multiples.
cudaError_t march_tensor_maps(const void* state, int nx, int ny, int pitch, int64_t plane,
                              TmaDesc* load, TmaDesc* store)
{
    static_assert(sizeof(TmaDesc) == sizeof(CUtensorMap), "opaque tensor map size");
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<Encode>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANE};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)plane * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t box_ld[3] = {RW, 2, NPLANE}, box_st[3] = {BW, 2, NPLANE};
    void* base = const_cast<void*>(state);
    if (encode(reinterpret_cast<CUtensorMap*>(load), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
               strides, box_ld, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (encode(reinterpret_cast<CUtensorMap*>(store), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
               strides, box_st, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_march(int mode, const ModelConst<float>& K, const StepLaunch& a, cudaStream_t s)
{
    int g, rows;
    march_plan(mode, K.nx, K.ny, &g, &rows);
    if (g < 0) return cudaErrorInvalidConfiguration;
    if (g != a.grid) return cudaErrorInvalidConfiguration; // partial buffers sized for a.grid
    const bool avg = a.stage >= 2;
    if (!a.tm_in || !a.tm_out) return cudaErrorInvalidValue;
    const bool srt = (mode & 4) != 0;
    switch (mode & 3) {
    case 0: launch_variant<0, false>(avg, srt, K, a, rows, s); break;
    case 1: launch_variant<1, false>(avg, srt, K, a, rows, s); break;
    case 2: launch_variant<0, true>(avg, srt, K, a, rows, s); break;
    default: launch_variant<1, true>(avg, srt, K, a, rows, s); break;
    }
    return cudaGetLastError();
}

} // namespace lbk
