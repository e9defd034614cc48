// api.cu -- the C ABI declared in include/lbkm.h.
//
// A handle owns two device copies of the state, laid out as 17 planes
// (f_1..f_16, lambda) of ny rows with a pitch that is a multiple of 32
// elements, plus the TNE partial buffer, the on-the-fly TNE history ring and a
// small block of device counters. lbkm_step launches one fused step kernel per
// time step; chunks of GRAPH_CHUNK steps are captured once into a CUDA graph
// and replayed, so control crosses from host to device once per chunk.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "lbkm.h"
#include "adjoint.cuh"
#include "kernels.cuh"
#include "model.h"

using namespace lbk;

namespace {
constexpr int GRAPH_CHUNK = 32; // even, so a replay leaves the ping-pong index unchanged
thread_local std::string g_create_error;
}

struct lbkm {
    lbkm_params p;
    HostModel hm;
    ModelConst<double> Kd;
    ModelConst<float> Kf;
    int precision, recovery;
    bool two_d;
    int nx, ny, pitch;
    size_t elem, plane_elems, state_bytes_dev;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    void* buf[2];
    void* buf3;  // the middle-stage state of the three-stage scheme (time_scheme 2)
    TmaDesc tm_load[3], tm_store[3]; // tensor maps of buf[0], buf[1], buf3 (FP32 2-D)
    int cur;
    int srt;     // the FP32 2-D step takes the single-relaxation-time fast path
    double* partials;
    int grid, tgrid;
    DevCounters* ctr;
    TneRecord* hist;
    TneRecord* tne_out;
    bool initialized;
    int64_t host_steps;
    cudaGraphExec_t graph[2];
    std::string err;
    // batched 1-D instances
    bool batched;
    int n_inst;
    std::vector<int32_t> inst_nx;
    InstParam* d_inst;
    BatchItem* d_items;
    int nitems;
    unsigned* d_bar;
    int bt;          // threads per block of the persistent kernel
    int bgrid;       // blocks of the persistent kernel
    long long wait_ns;
    int phantom;
    TneRecord* d_inst_tne;
};

namespace {

lbkm_status fail(lbkm_t h, lbkm_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CUDA_TRY(h, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), e_ == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

const void* model_ptr(const lbkm* h)
{
    return h->precision == 0 ? (const void*)&h->Kd : (const void*)&h->Kf;
}

// stage 0: Euler step buf[from] -> buf[1-from]; stage 1: first Runge-Kutta stage, same
// buffers (u1 = E(u^n) into buf[1-from]); stage 2: last stage from `src` (u1 for RK2, u2
// for RK3) back into buf[from] with weights (wp, wn) on (u^n, E(src)); stage 3: the
// middle RK3 stage, u2 = 3/4 u^n + 1/4 E(u1) into buf3
// Device memory of a handle: the caller's allocator (lbkm_params.alloc / free, with the
// handle's stream) when it set one, else cudaMalloc / cudaFree.
cudaError_t dmalloc(const lbkm* h, void** ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (!h->p.alloc) return cudaMalloc(ptr, bytes);
    void* q = h->p.alloc(bytes, (void*)h->stream, h->p.alloc_ctx);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) & 255u) {
        h->p.free(q, (void*)h->stream, h->p.alloc_ctx);
        return cudaErrorMisalignedAddress;
    }
    *ptr = q;
    return cudaSuccess;
}
template <typename T>
cudaError_t dmalloc(const lbkm* h, T** ptr, size_t bytes)
{
    return dmalloc(h, reinterpret_cast<void**>(ptr), bytes);
}
void dfree(const lbkm* h, void* ptr)
{
    if (!ptr) return;
    if (h->p.alloc)
        h->p.free(ptr, (void*)h->stream, h->p.alloc_ctx);
    else
        cudaFree(ptr);
}
// Page-locked host memory mapped into the device's address space at the same address
// (any pinned buffer under unified addressing): kernels read or write it in place.
bool device_addressable_host(const void* p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}
// a temporary of one call: freed (after its stream has drained) when the call returns
struct DevTemp {
    const lbkm* h;
    void* p = nullptr;
    explicit DevTemp(const lbkm* hh) : h(hh) {}
    ~DevTemp()
    {
        if (p) {
            cudaStreamSynchronize(h->stream);
            dfree(h, p);
        }
    }
};

StepLaunch step_args(const lbkm* h, int from, int stage = 0, const void* src = nullptr,
                     double wp = 0.0, double wn = 1.0)
{
    StepLaunch a;
    a.in = stage >= 2 ? src : h->buf[from];
    a.out = stage == 2 ? h->buf[from] : (stage == 3 ? h->buf3 : h->buf[1 - from]);
    a.prev = h->buf[from];
    a.stage = stage;
    a.wprev = wp;
    a.wnew = wn;
    a.partials = h->partials;
    a.ctr = h->ctr;
    a.hist = h->hist;
    a.hist_cap = h->p.tne_capacity;
    a.tne_every = h->p.tne_every;
    a.grid = h->grid;
    a.cell_area = h->p.dx * h->p.dy;
    auto map_of = [&](const void* b) { return b == h->buf[0] ? 0 : (b == h->buf[1] ? 1 : 2); };
    a.tm_in = &h->tm_load[map_of(a.in)];
    a.tm_out = &h->tm_store[map_of(a.out)];
    a.srt = h->srt;
    return a;
}

lbkm_status check_status(lbkm_t h)
{
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int st = 0;
    CUDA_TRY(h, cudaMemcpy(&st, &h->ctr->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 2)
        return fail(h, LBKM_ETIMEOUT,
                    "a grid barrier wait of the persistent kernel ran out of time");
    if (st & 1)
        return fail(h, LBKM_EUNSTABLE,
                    "a cell reached a non-finite or non-positive density or temperature");
    return LBKM_OK;
}

void release(lbkm* h)
{
    for (int i = 0; i < 2; i++)
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    dfree(h, h->buf[0]);
    dfree(h, h->buf[1]);
    dfree(h, h->buf3);
    dfree(h, h->partials);
    dfree(h, h->ctr);
    dfree(h, h->hist);
    dfree(h, h->tne_out);
    dfree(h, h->d_inst);
    dfree(h, h->d_items);
    dfree(h, h->d_bar);
    dfree(h, h->d_inst_tne);
}

// Work items of the batched kernel for segments of `seg` cells.
cudaError_t build_items(lbkm* h, int seg)
{
    std::vector<BatchItem> items;
    for (int i = 0; i < h->n_inst; i++)
        for (int x0 = 0; x0 < h->inst_nx[i]; x0 += seg) items.push_back({i, x0});
    dfree(h, h->d_items);
    h->d_items = nullptr;
    cudaError_t e = dmalloc(h, &h->d_items, sizeof(BatchItem) * items.size());
    if (e != cudaSuccess) return e;
    h->nitems = (int)items.size();
    return cudaMemcpy(h->d_items, items.data(), sizeof(BatchItem) * items.size(),
                      cudaMemcpyHostToDevice);
}

BatchLaunch batch_args(const lbkm* h, int nsteps)
{
    BatchLaunch b;
    b.buf[0] = h->buf[0];
    b.buf[1] = h->buf[1];
    b.cur = h->cur;
    b.inst = h->d_inst;
    b.items = h->d_items;
    b.nitems = h->nitems;
    b.ctr = h->ctr;
    b.bar = h->d_bar;
    b.nsteps = nsteps;
    b.phantom_blocks = h->phantom;
    b.wait_ns = h->wait_ns;
    return b;
}

} // namespace

extern "C" {

void lbkm_default_params(lbkm_params* p)
{
    memset(p, 0, sizeof(*p));
    p->precision = LBKM_F64;
    p->recovery = LBKM_RECOVER_F64;
    p->gamma = 1.4;
    p->Pr = 0.0;
    const int32_t kind[4] = {0, 1, 0, 1};
    const double speed[4] = {2.7, 2.2, 1.2, 1.0}, eta[4] = {5.0, 0.0, 3.0, 0.0};
    for (int o = 0; o < 4; o++) {
        p->orbit_kind[o] = kind[o];
        p->orbit_speed[o] = speed[o];
        p->orbit_eta[o] = eta[o];
    }
    for (int k = 0; k < 16; k++) p->S[k] = 1e5;
    p->T_ig = 1.1;
    p->dx = p->dy = 1e-3;
    p->dt = 1e-5;
    p->bc_x = LBKM_BC_ZERO_GRADIENT;
    p->bc_y = LBKM_BC_PERIODIC;
    p->tne_capacity = 1;
}

// f_hat^eq_1..16 of (rho, u, T) (list after Eq. (16), entries 14 and 16 per Eq. (11)),
// for the fixed ghost values of Dirichlet sides
static void host_feq_moments(double DI, double rho, double ux, double uy, double T, double* q)
{
    const double u2 = ux * ux + uy * uy, A = (DI + 2) * T + u2, B = (DI + 4) * T + u2;
    q[0] = rho;
    q[1] = rho * ux;
    q[2] = rho * uy;
    q[3] = rho * (DI * T + u2);
    q[4] = rho * (T + ux * ux);
    q[5] = rho * ux * uy;
    q[6] = rho * (T + uy * uy);
    q[7] = rho * ux * A;
    q[8] = rho * uy * A;
    q[9] = 3 * rho * ux * T + rho * ux * ux * ux;
    q[10] = rho * uy * T + rho * ux * ux * uy;
    q[11] = rho * ux * T + rho * ux * uy * uy;
    q[12] = 3 * rho * uy * T + rho * uy * uy * uy;
    q[13] = rho * A * T + rho * ux * ux * B;
    q[14] = rho * ux * uy * B;
    q[15] = rho * A * T + rho * uy * uy * B;
}

lbkm_status lbkm_create(const lbkm_params* pin, void* cuda_stream, lbkm_t* out)
{
    if (!out) return fail(nullptr, LBKM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!pin) return fail(nullptr, LBKM_EINVAL, "params is NULL");
    lbkm_params p = *pin;
    if (p.nx < 1 || p.ny < 1) return fail(nullptr, LBKM_EINVAL, "nx and ny must be >= 1");
    if (p.nx > (1 << 28) || p.ny > (1 << 28) || (double)p.nx * p.ny > 4e9)
        return fail(nullptr, LBKM_EINVAL, "grid too large");
    if (p.precision != LBKM_F64 && p.precision != LBKM_F32)
        return fail(nullptr, LBKM_EINVAL, "precision must be LBKM_F64 or LBKM_F32");
    if (p.recovery != LBKM_RECOVER_F64 && p.recovery != LBKM_RECOVER_DF32)
        return fail(nullptr, LBKM_EINVAL, "recovery must be LBKM_RECOVER_F64 or _DF32");
    if (!(p.gamma > 1.0 && p.gamma <= 2.0))
        return fail(nullptr, LBKM_EINVAL, "gamma must lie in (1, 2] (I = 2/(gamma-1) - 2 >= 0)");
    for (int o = 0; o < 4; o++) {
        if (!(p.orbit_speed[o] > 0.0)) return fail(nullptr, LBKM_EINVAL, "orbit_speed must be > 0");
        if (!(p.orbit_eta[o] >= 0.0)) return fail(nullptr, LBKM_EINVAL, "orbit_eta must be >= 0");
    }
    if (!(p.dx > 0 && p.dy > 0 && p.dt > 0))
        return fail(nullptr, LBKM_EINVAL, "dx, dy, dt must be > 0");
    if (!(p.bc_x == LBKM_BC_PERIODIC || p.bc_x == LBKM_BC_ZERO_GRADIENT || p.bc_x == LBKM_BC_SIDES) ||
        !(p.bc_y == LBKM_BC_PERIODIC || p.bc_y == LBKM_BC_ZERO_GRADIENT || p.bc_y == LBKM_BC_WALL ||
          p.bc_y == LBKM_BC_SIDES))
        return fail(nullptr, LBKM_EINVAL,
                    "bc_x must be LBKM_BC_PERIODIC, _ZERO_GRADIENT or _SIDES; bc_y one of those "
                    "or _WALL");
    int sbc[4];
    for (int s = 0; s < 4; s++) {
        const int dir = s < 2 ? p.bc_x : p.bc_y;
        sbc[s] = dir == LBKM_BC_SIDES ? p.side_bc[s] : dir;
        const bool x_side = s < 2;
        const bool ok = sbc[s] == LBKM_BC_PERIODIC ? dir != LBKM_BC_SIDES
                        : sbc[s] == LBKM_BC_ZERO_GRADIENT || sbc[s] == LBKM_BC_DIRICHLET
                            ? true
                            : (sbc[s] == LBKM_BC_WALL || sbc[s] == LBKM_BC_SPECULAR) && !x_side;
        if (!ok)
            return fail(nullptr, LBKM_EINVAL,
                        "side %d: periodic only for both sides, walls and specular only in y", s);
        if (!x_side && p.ny < 2 && sbc[s] >= LBKM_BC_WALL)
            return fail(nullptr, LBKM_EINVAL, "walls, Dirichlet or specular y sides need ny >= 2");
        if (sbc[s] == LBKM_BC_WALL) {
            const int w = s - 2;
            if (!(p.wall_T[w] > 0.0 && p.wall_T[w] < 1e300) || !(fabs(p.wall_ux[w]) < 1e300) ||
                !(fabs(p.wall_uy[w]) < 1e300))
                return fail(nullptr, LBKM_EINVAL, "wall velocities must be finite, wall_T > 0");
        }
        if (sbc[s] == LBKM_BC_DIRICHLET &&
            (!(p.side_rho[s] > 0.0 && p.side_rho[s] < 1e300) ||
             !(p.side_T[s] > 0.0 && p.side_T[s] < 1e300) || !(fabs(p.side_ux[s]) < 1e300) ||
             !(fabs(p.side_uy[s]) < 1e300) || !(p.side_lam[s] >= 0.0 && p.side_lam[s] <= 1.0)))
            return fail(nullptr, LBKM_EINVAL,
                        "Dirichlet side %d: rho, T > 0 and finite u, lambda in [0, 1]", s);
    }
    if (p.Pr > 0) p.S[7] = p.S[8] = p.Pr * p.S[4];
    double smax = 0;
    for (int k = 4; k < 16; k++) {
        if (!(p.S[k] > 0)) return fail(nullptr, LBKM_EINVAL, "S_%d must be > 0", k + 1);
        if (p.S[k] > smax) smax = p.S[k];
    }
    if (!(p.dt * smax < 2.0))
        return fail(nullptr, LBKM_EINVAL,
                    "dt * max(S_5..S_16) = %g: forward Euler relaxation needs < 2", p.dt * smax);
    double vmax = 0;
    for (int o = 0; o < 4; o++) vmax = fmax(vmax, p.orbit_speed[o]);
    double cfl = vmax * p.dt * (1.0 / p.dx + (p.ny > 1 ? 1.0 / p.dy : 0.0));
    if (!(cfl <= 1.0))
        return fail(nullptr, LBKM_EINVAL, "CFL number %g of the fastest velocity exceeds 1", cfl);
    if (!(p.omega1 >= 0 && p.omega2 >= 0))
        return fail(nullptr, LBKM_EINVAL, "omega1, omega2 must be >= 0");
    if (!(p.T_ig >= 0.0 && p.T_ig <= 1e300))
        return fail(nullptr, LBKM_EINVAL, "T_ig must be finite and >= 0");
    if (p.time_scheme < 0 || p.time_scheme > 2)
        return fail(nullptr, LBKM_EINVAL,
                    "time_scheme must be 0 (Euler), 1 (SSP-RK2) or 2 (SSP-RK3)");
    if (p.tne_every < 0 || p.tne_capacity < 1)
        return fail(nullptr, LBKM_EINVAL, "tne_every must be >= 0 and tne_capacity >= 1");
    if (p.collision != 0 && p.collision != 1)
        return fail(nullptr, LBKM_EINVAL, "collision must be 0 (fast path where it applies) or 1");
    if ((p.alloc == nullptr) != (p.free == nullptr))
        return fail(nullptr, LBKM_EINVAL, "alloc and free must be set together");

    lbkm* h = new lbkm();
    h->p = p;
    char err[256] = {0};
    if (build_host_model(p.orbit_kind, p.orbit_speed, p.orbit_eta, p.gamma, &h->hm, err,
                         sizeof(err)) != 0) {
        delete h;
        bool kind = strstr(err, "orbit_kind") != nullptr;
        return fail(nullptr, kind ? LBKM_EINVAL : LBKM_ESINGULAR, "%s", err);
    }
    h->precision = p.precision;
    h->recovery = p.recovery;
    h->two_d = p.ny > 1;
    h->nx = p.nx;
    h->ny = p.ny;
    h->pitch = (p.nx + 31) / 32 * 32;
    h->elem = p.precision == LBKM_F64 ? 8 : 4;
    h->plane_elems = (size_t)h->ny * h->pitch;
    h->state_bytes_dev = (size_t)NPLANE * h->plane_elems * h->elem;
    fill_model_const<double>(h->hm, p.S, p.Q, p.omega1, p.omega2, p.T_ig, p.dx, p.dy, p.dt, p.nx,
                             p.ny, h->pitch, p.bc_x, p.bc_y, &h->Kd);
    fill_model_const<float>(h->hm, p.S, p.Q, p.omega1, p.omega2, p.T_ig, p.dx, p.dy, p.dt, p.nx,
                            p.ny, h->pitch, p.bc_x, p.bc_y, &h->Kf);
    // per-side conditions; Dirichlet ghost values f = M^-1 f_hat^eq(state), lambda
    for (int sd = 0; sd < 4; sd++) {
        h->Kd.sbc[sd] = h->Kf.sbc[sd] = sbc[sd];
        if (sbc[sd] != LBKM_BC_DIRICHLET) continue;
        double fe[16];
        host_feq_moments(2.0 + h->hm.I, p.side_rho[sd], p.side_ux[sd], p.side_uy[sd], p.side_T[sd],
                         fe);
        for (int i = 0; i < 16; i++) {
            double acc = 0.0;
            for (int k = 0; k < 16; k++) acc += h->hm.Minv[i * 16 + k] * fe[k];
            h->Kd.sfeq[sd][i] = acc;
            h->Kf.sfeq[sd][i] = (float)acc;
        }
        h->Kd.sfeq[sd][16] = p.side_lam[sd];
        h->Kf.sfeq[sd][16] = (float)p.side_lam[sd];
    }
    for (int side = 0; side < 2; side++) {
        h->Kd.wux[side] = p.wall_ux[side];
        h->Kd.wuy[side] = p.wall_uy[side];
        h->Kd.wT[side] = p.wall_T[side];
        h->Kf.wux[side] = (float)p.wall_ux[side];
        h->Kf.wuy[side] = (float)p.wall_uy[side];
        h->Kf.wT[side] = (float)p.wall_T[side];
    }
    h->stream = (cudaStream_t)cuda_stream;

    auto bail = [&](cudaError_t e, const char* what) {
        std::string m = std::string(what) + ": " +
                        (e == cudaErrorMisalignedAddress ? "alloc returned a block not aligned to 256 bytes"
                                                         : cudaGetErrorString(e));
        release(h);
        delete h;
        return fail(nullptr,
                    e == cudaErrorMemoryAllocation ? LBKM_ENOMEM
                    : e == cudaErrorMisalignedAddress ? LBKM_EINVAL : LBKM_ECUDA,
                    "%s", m.c_str());
    };
    cudaError_t e;
    if ((e = dmalloc(h, &h->buf[0], h->state_bytes_dev)) != cudaSuccess) return bail(e, "state A");
    if ((e = dmalloc(h, &h->buf[1], h->state_bytes_dev)) != cudaSuccess) return bail(e, "state B");
    if ((e = cudaMemset(h->buf[0], 0, h->state_bytes_dev)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemset(h->buf[1], 0, h->state_bytes_dev)) != cudaSuccess) return bail(e, "memset");
    if (p.time_scheme == 2) {
        if ((e = dmalloc(h, &h->buf3, h->state_bytes_dev)) != cudaSuccess) return bail(e, "state C");
        if ((e = cudaMemset(h->buf3, 0, h->state_bytes_dev)) != cudaSuccess) return bail(e, "memset");
    }
    // single-relaxation-time fast path (Sec. V, Eq. (87)): equal R_5..R_16, no TNE,
    // forward Euler, FP32 2-D, periodic or zero-gradient sides
    bool equal = true;
    for (int k = 5; k < 16; k++) equal = equal && p.S[k] == p.S[4];
    h->srt = (p.collision == 0 && equal && p.tne_every == 0 && p.time_scheme == 0 &&
              h->precision == LBKM_F32 && h->two_d && sbc[0] <= 1 && sbc[1] <= 1 && sbc[2] <= 1 &&
              sbc[3] <= 1)
                 ? 1 : 0;
    if (h->precision == LBKM_F32 && h->two_d) {
        void* bufs[3] = {h->buf[0], h->buf[1], h->buf3};
        for (int b = 0; b < 3; b++) {
            if (!bufs[b]) continue;
            e = march_tensor_maps(bufs[b], h->nx, h->ny, h->pitch, (int64_t)h->plane_elems,
                                  &h->tm_load[b], &h->tm_store[b]);
            if (e != cudaSuccess) return bail(e, "tensor maps");
        }
    }
    h->grid = step_grid(h->precision, h->recovery, h->two_d, h->nx, h->ny, sbc);
    if (h->grid < 1) return bail(cudaGetLastError(), "step grid");
    h->tgrid = tne_grid(h->nx, h->ny);
    int pg = h->grid > h->tgrid ? h->grid : h->tgrid;
    if ((e = dmalloc(h, &h->partials, sizeof(double) * TNE_PART * (size_t)pg)) != cudaSuccess)
        return bail(e, "partials");
    if ((e = dmalloc(h, &h->ctr, sizeof(DevCounters))) != cudaSuccess) return bail(e, "counters");
    if ((e = cudaMemset(h->ctr, 0, sizeof(DevCounters))) != cudaSuccess) return bail(e, "memset");
    if ((e = dmalloc(h, &h->hist, sizeof(TneRecord) * (size_t)p.tne_capacity)) != cudaSuccess)
        return bail(e, "history");
    if ((e = dmalloc(h, &h->tne_out, sizeof(TneRecord))) != cudaSuccess) return bail(e, "tne out");
    if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "capture stream");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "synchronize");
    *out = h;
    return LBKM_OK;
}

void lbkm_destroy(lbkm_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

lbkm_status lbkm_set_stream(lbkm_t h, void* s)
{
    if (!h) return LBKM_EINVAL;
    h->stream = (cudaStream_t)s;
    return LBKM_OK;
}

lbkm_status lbkm_init_fields(lbkm_t h, const double* rho, const double* ux, const double* uy,
                             const double* T, const double* lambda, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!rho || !ux || !uy || !T) return fail(h, LBKM_EINVAL, "rho, ux, uy and T are required");
    const size_t n = (size_t)h->nx * h->ny, nb = n * sizeof(double);
    DevTemp tt(h);
    double* tmp = nullptr;
    const double *r = rho, *u = ux, *v = uy, *t = T, *l = lambda;
    // pinned host fields are read by the kernel in place
    const bool in_place = on_device || (device_addressable_host(rho) && device_addressable_host(ux) &&
                                        device_addressable_host(uy) && device_addressable_host(T) &&
                                        device_addressable_host(lambda));
    if (!in_place) {
        CUDA_TRY(h, dmalloc(h, &tt.p, nb * 5));
        tmp = static_cast<double*>(tt.p);
        const double* src[5] = {rho, ux, uy, T, lambda};
        for (int k = 0; k < 5; k++) {
            if (!src[k]) continue;
            CUDA_TRY(h, cudaMemcpyAsync(tmp + k * n, src[k], nb, cudaMemcpyHostToDevice, h->stream));
        }
        r = tmp;
        u = tmp + n;
        v = tmp + 2 * n;
        t = tmp + 3 * n;
        l = lambda ? tmp + 4 * n : nullptr;
    }
    h->cur = 0;
    CUDA_TRY(h, launch_init(h->precision, h->Kd, r, u, v, t, l, h->buf[0], h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->initialized = true;
    h->host_steps = 0;
    return LBKM_OK;
}

// One time step from buf[c]: forward Euler (one launch, the state moves to the other
// buffer), or the two-stage SSP Runge-Kutta scheme (E(u^n) into the other buffer, then
// (u^n + E(E(u^n))) / 2 back into buf[c]). c is updated to the buffer holding u^{n+1}.
// With TNE on, a small kernel then turns the step's per-block partials into the record.
// The three-stage scheme (Shu and Osher's SSP-RK3): u1 = E(u^n) into buf[1-c],
// u2 = 3/4 u^n + 1/4 E(u1) into buf3, u^{n+1} = 1/3 u^n + 2/3 E(u2) back into buf[c].
static cudaError_t launch_full_step(const lbkm* h, const void* K, int& c, cudaStream_t st)
{
    const int ts = h->p.time_scheme;
    const StepLaunch a0 = step_args(h, c, ts == 0 ? 0 : 1);
    cudaError_t e = launch_step(h->precision, h->recovery, h->two_d, K, a0, st);
    if (e == cudaSuccess && ts == 1)
        e = launch_step(h->precision, h->recovery, h->two_d, K,
                        step_args(h, c, 2, h->buf[1 - c], 0.5, 0.5), st);
    if (e == cudaSuccess && ts == 2) {
        e = launch_step(h->precision, h->recovery, h->two_d, K,
                        step_args(h, c, 3, h->buf[1 - c], 0.75, 0.25), st);
        if (e == cudaSuccess)
            e = launch_step(h->precision, h->recovery, h->two_d, K,
                            step_args(h, c, 2, h->buf3, 1.0 / 3.0, 2.0 / 3.0), st);
    }
    if (e == cudaSuccess && a0.tne_every > 0) e = launch_tne_finish(a0, st);
    if (e == cudaSuccess && ts == 0) c = 1 - c;
    return e;
}

lbkm_status lbkm_step(lbkm_t h, int64_t n)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_step before lbkm_init_fields");
    if (n < 0) return fail(h, LBKM_EINVAL, "n must be >= 0");
    if (h->batched) {
        // one persistent launch per chunk of steps, replayed from a CUDA graph
        while (n >= GRAPH_CHUNK) {
            cudaGraphExec_t& ex = h->graph[h->cur];
            if (!ex) {
                cudaGraph_t g;
                CUDA_TRY(h, cudaStreamBeginCapture(h->capture_stream,
                                                   cudaStreamCaptureModeThreadLocal));
                cudaError_t le = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned),
                                                 h->capture_stream);
                if (le == cudaSuccess)
                    le = launch_batch(h->recovery, h->bt, h->Kf, batch_args(h, GRAPH_CHUNK),
                                      h->bgrid, h->capture_stream);
                cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
                if (le != cudaSuccess || ce != cudaSuccess) {
                    if (ce == cudaSuccess) cudaGraphDestroy(g);
                    return fail(h, LBKM_ECUDA, "graph capture of the persistent kernel: %s",
                                cudaGetErrorString(le != cudaSuccess ? le : ce));
                }
                cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess)
                    return fail(h, LBKM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            CUDA_TRY(h, cudaGraphLaunch(ex, h->stream));
            n -= GRAPH_CHUNK;
            h->host_steps += GRAPH_CHUNK;
        }
        if (n > 0) {
            CUDA_TRY(h, cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
            CUDA_TRY(h, launch_batch(h->recovery, h->bt, h->Kf, batch_args(h, (int)n), h->bgrid,
                                     h->stream));
            h->cur ^= (int)(n & 1);
            h->host_steps += n;
        }
        return LBKM_OK;
    }
    const void* K = model_ptr(h);
    while (n >= GRAPH_CHUNK) {
        cudaGraphExec_t& ex = h->graph[h->cur];
        if (!ex) {
            cudaGraph_t g;
            CUDA_TRY(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
            int c = h->cur;
            cudaError_t le = cudaSuccess;
            for (int s = 0; s < GRAPH_CHUNK && le == cudaSuccess; s++)
                le = launch_full_step(h, K, c, h->capture_stream);
            cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
            if (le != cudaSuccess || ce != cudaSuccess) {
                if (ce == cudaSuccess) cudaGraphDestroy(g);
                return fail(h, LBKM_ECUDA, "graph capture: %s",
                            cudaGetErrorString(le != cudaSuccess ? le : ce));
            }
            cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess)
                return fail(h, LBKM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
        }
        CUDA_TRY(h, cudaGraphLaunch(ex, h->stream));
        n -= GRAPH_CHUNK;
        h->host_steps += GRAPH_CHUNK;
    }
    for (; n > 0; n--) {
        CUDA_TRY(h, launch_full_step(h, K, h->cur, h->stream));
        h->host_steps++;
    }
    return LBKM_OK;
}

lbkm_status lbkm_sync(lbkm_t h)
{
    if (!h) return LBKM_EINVAL;
    return check_status(h);
}

int64_t lbkm_steps_taken(lbkm_t h) { return h ? h->host_steps : -1; }

lbkm_status lbkm_macros(lbkm_t h, double* rho, double* ux, double* uy, double* T, double* p,
                        double* lambda, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_macros before lbkm_init_fields");
    const size_t n = (size_t)h->nx * h->ny, nb = n * sizeof(double);
    double* outs[6] = {rho, ux, uy, T, p, lambda};
    double* dev[6] = {rho, ux, uy, T, p, lambda};
    DevTemp tt(h);
    // pinned host outputs are written by the kernel in place
    bool in_place = on_device;
    if (!in_place) {
        in_place = true;
        for (int k = 0; k < 6; k++) in_place = in_place && device_addressable_host(outs[k]);
    }
    if (!in_place) {
        CUDA_TRY(h, dmalloc(h, &tt.p, nb * 6));
        double* tmp = static_cast<double*>(tt.p);
        for (int k = 0; k < 6; k++) dev[k] = outs[k] ? tmp + k * n : nullptr;
    }
    CUDA_TRY(h, launch_macros(h->precision, h->Kd, h->buf[h->cur], dev[0], dev[1], dev[2], dev[3],
                              dev[4], dev[5], h->stream));
    if (!in_place) {
        for (int k = 0; k < 6; k++)
            if (outs[k])
                CUDA_TRY(h, cudaMemcpyAsync(outs[k], dev[k], nb, cudaMemcpyDeviceToHost, h->stream));
    }
    return check_status(h);
}

static void record_to_global(const TneRecord& r, lbkm_tne_global* g)
{
    memcpy(g->sum, r.sum, sizeof(g->sum));
    memcpy(g->abs_sum, r.abs_sum, sizeof(g->abs_sum));
    memcpy(g->min, r.min, sizeof(g->min));
    memcpy(g->max, r.max, sizeof(g->max));
    g->d_sum = r.d_sum;
    g->d2_sum = r.d2_sum;
    g->step = r.step;
}

lbkm_status lbkm_tne(lbkm_t h, double* delta, lbkm_tne_global* g, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_tne before lbkm_init_fields");
    const size_t n = (size_t)h->nx * h->ny, nb = 16 * n * sizeof(double);
    double* dd = delta;
    DevTemp tt(h);
    double* tmp = nullptr;
    if (delta && !on_device) {
        CUDA_TRY(h, dmalloc(h, &tt.p, nb));
        tmp = dd = static_cast<double*>(tt.p);
    }
    CUDA_TRY(h, launch_tne(h->precision, h->Kd, h->buf[h->cur], dd, h->partials, h->tgrid, h->ctr,
                           h->tne_out, h->p.dx * h->p.dy, h->stream));
    if (tmp) {
        CUDA_TRY(h, cudaMemcpyAsync(delta, tmp, nb, cudaMemcpyDeviceToHost, h->stream));
    }
    TneRecord r;
    CUDA_TRY(h, cudaMemcpyAsync(&r, h->tne_out, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    lbkm_status st = check_status(h);
    if (st != LBKM_OK) return st;
    if (g) record_to_global(r, g);
    return LBKM_OK;
}

lbkm_status lbkm_tne_history(lbkm_t h, lbkm_tne_global* out, int32_t max_records, int32_t* n_out)
{
    if (!h || !n_out || (max_records > 0 && !out)) return LBKM_EINVAL;
    *n_out = 0;
    lbkm_status st = check_status(h);
    if (st != LBKM_OK) return st;
    DevCounters c;
    CUDA_TRY(h, cudaMemcpy(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost));
    const int cap = h->p.tne_capacity;
    int64_t have = c.hist_count < cap ? c.hist_count : cap;
    int64_t take = have < max_records ? have : max_records;
    if (take > 0) {
        // the oldest records kept, in order: one copy up to the ring's end, one after it
        std::vector<TneRecord> r((size_t)take);
        const int64_t start = (c.hist_count - have) % cap;
        const int64_t n1 = take < cap - start ? take : cap - start;
        CUDA_TRY(h, cudaMemcpy(r.data(), h->hist + start, sizeof(TneRecord) * n1,
                               cudaMemcpyDeviceToHost));
        if (take > n1)
            CUDA_TRY(h, cudaMemcpy(r.data() + n1, h->hist, sizeof(TneRecord) * (take - n1),
                                   cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < take; k++) record_to_global(r[k], out + k);
    }
    *n_out = (int32_t)take;
    return LBKM_OK;
}

size_t lbkm_state_bytes(lbkm_t h)
{
    if (!h) return 0;
    return (size_t)NPLANE * h->nx * h->ny * h->elem + sizeof(int64_t);
}

lbkm_status lbkm_get_state(lbkm_t h, void* dst, int on_device)
{
    if (!h || !dst) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_get_state before lbkm_init_fields");
    const size_t row = (size_t)h->nx * h->elem, plane = row * h->ny;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int pl = 0; pl < NPLANE; pl++)
        CUDA_TRY(h, cudaMemcpy2DAsync((char*)dst + pl * plane, row,
                                      (char*)h->buf[h->cur] + pl * h->plane_elems * h->elem,
                                      h->pitch * h->elem, row, h->ny, k, h->stream));
    int64_t s = h->host_steps;
    CUDA_TRY(h, cudaMemcpyAsync((char*)dst + NPLANE * plane, &s, sizeof(s),
                                on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                                h->stream));
    return check_status(h);
}

lbkm_status lbkm_set_state(lbkm_t h, const void* src, int on_device)
{
    if (!h || !src) return LBKM_EINVAL;
    const size_t row = (size_t)h->nx * h->elem, plane = row * h->ny;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    h->cur = 0;
    for (int pl = 0; pl < NPLANE; pl++)
        CUDA_TRY(h, cudaMemcpy2DAsync((char*)h->buf[0] + pl * h->plane_elems * h->elem,
                                      h->pitch * h->elem, (const char*)src + pl * plane, row, row,
                                      h->ny, k, h->stream));
    int64_t s = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&s, (const char*)src + NPLANE * plane, sizeof(s),
                                on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    DevCounters c;
    memset(&c, 0, sizeof(c));
    c.step = s;
    CUDA_TRY(h, cudaMemcpy(h->ctr, &c, sizeof(c), cudaMemcpyHostToDevice));
    h->host_steps = s;
    h->initialized = true;
    return LBKM_OK;
}

lbkm_status lbkm_create_batched(const lbkm_params* pin, int32_t n_instances,
                                const int32_t* inst_nx, const double* inst_S,
                                const double* inst_Q, const double* inst_omega1,
                                void* cuda_stream, lbkm_t* out)
{
    if (!out) return fail(nullptr, LBKM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!pin || !inst_nx || n_instances < 1)
        return fail(nullptr, LBKM_EINVAL, "params, inst_nx and n_instances >= 1 are required");
    if (pin->precision != LBKM_F32)
        return fail(nullptr, LBKM_EINVAL, "batched instances run in LBKM_F32");
    if (pin->time_scheme != 0)
        return fail(nullptr, LBKM_EINVAL, "batched instances step with forward Euler");
    if (pin->tne_every != 0)
        return fail(nullptr, LBKM_EINVAL,
                    "tne_every must be 0 for batched instances (use lbkm_tne_instances)");
    int64_t total = 0;
    for (int i = 0; i < n_instances; i++) {
        if (inst_nx[i] < 4 || inst_nx[i] % 4 != 0)
            return fail(nullptr, LBKM_EINVAL, "instance %d: nx must be a multiple of 4 and >= 4",
                        i);
        total += inst_nx[i];
    }
    if (total > (1 << 28)) return fail(nullptr, LBKM_EINVAL, "too many cells in total");
    lbkm_params q = *pin;
    q.nx = (int32_t)total;
    q.ny = 1;
    q.bc_x = LBKM_BC_ZERO_GRADIENT;
    q.bc_y = LBKM_BC_PERIODIC;
    std::vector<InstParam> ip(n_instances);
    const double DI = 2.0 + (2.0 / (pin->gamma - 1.0) - 2.0);
    int64_t off = 0;
    for (int i = 0; i < n_instances; i++) {
        double S[16];
        for (int k = 0; k < 16; k++) S[k] = inst_S ? inst_S[16 * i + k] : pin->S[k];
        if (pin->Pr > 0) S[7] = S[8] = pin->Pr * S[4];
        double smax = 0;
        for (int k = 4; k < 16; k++) {
            if (!(S[k] > 0)) return fail(nullptr, LBKM_EINVAL, "instance %d: S must be > 0", i);
            smax = fmax(smax, S[k]);
        }
        if (!(pin->dt * smax < 2.0))
            return fail(nullptr, LBKM_EINVAL, "instance %d: dt * max S = %g must be < 2", i,
                        pin->dt * smax);
        const double Q = inst_Q ? inst_Q[i] : pin->Q;
        const double om1 = inst_omega1 ? inst_omega1[i] : pin->omega1;
        if (!(om1 >= 0)) return fail(nullptr, LBKM_EINVAL, "instance %d: omega1 < 0", i);
        for (int k = 0; k < 16; k++) ip[i].S[k] = (float)S[k];
        ip[i].A8c = (float)((S[4] - S[7]) / S[4]);
        ip[i].A9c = (float)((S[6] - S[8]) / S[6]);
        ip[i].chem = (float)(2.0 * Q / (DI * pin->dt));
        ip[i].om1 = (float)om1;
        ip[i].om2 = (float)pin->omega2;
        ip[i].nx = inst_nx[i];
        ip[i].off = off;
        off += inst_nx[i];
    }
    lbkm_t h = nullptr;
    lbkm_status st = lbkm_create(&q, cuda_stream, &h);
    if (st != LBKM_OK) return st;
    h->batched = true;
    h->n_inst = n_instances;
    h->inst_nx.assign(inst_nx, inst_nx + n_instances);
    h->wait_ns = 2000000000LL;
    h->phantom = 0;
    cudaError_t e = dmalloc(h, &h->d_inst, sizeof(InstParam) * n_instances);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_inst, ip.data(), sizeof(InstParam) * n_instances,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dmalloc(h, &h->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->d_bar, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = dmalloc(h, &h->d_inst_tne, sizeof(TneRecord) * n_instances);
    int sms = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    h->bt = 128;
    const int per_sm = batch_max_blocks(h->recovery, h->bt);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    h->bgrid = per_sm * sms;
    if (e == cudaSuccess) e = build_items(h, batch_segment(h->bt));
    if (e != cudaSuccess) {
        std::string m = cudaGetErrorString(e);
        lbkm_destroy(h);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA,
                    "batched set-up: %s", m.c_str());
    }
    *out = h;
    return LBKM_OK;
}

int32_t lbkm_instances(lbkm_t h) { return h ? (h->batched ? h->n_inst : 1) : 0; }

lbkm_status lbkm_tne_instances(lbkm_t h, lbkm_tne_global* out)
{
    if (!h || !out) return LBKM_EINVAL;
    if (!h->batched) return fail(h, LBKM_EINVAL, "lbkm_tne_instances needs a batched handle");
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_tne_instances before init");
    CUDA_TRY(h, launch_tne_instances(h->precision, h->Kd, h->buf[h->cur], h->d_inst, h->n_inst,
                                     h->d_inst_tne, h->p.dx * h->p.dy, h->stream));
    std::vector<TneRecord> r(h->n_inst);
    CUDA_TRY(h, cudaMemcpyAsync(r.data(), h->d_inst_tne, sizeof(TneRecord) * h->n_inst,
                                cudaMemcpyDeviceToHost, h->stream));
    lbkm_status st = check_status(h);
    if (st != LBKM_OK) return st;
    for (int i = 0; i < h->n_inst; i++) record_to_global(r[i], out + i);
    return LBKM_OK;
}

static void drop_graphs(lbkm_t h)
{
    for (int i = 0; i < 2; i++)
        if (h->graph[i]) {
            cudaGraphExecDestroy(h->graph[i]);
            h->graph[i] = nullptr;
        }
}

lbkm_status lbkm_set_wait_limit(lbkm_t h, int64_t timeout_ns, int32_t phantom_blocks)
{
    if (!h || timeout_ns < 1 || phantom_blocks < 0) return LBKM_EINVAL;
    h->wait_ns = timeout_ns;
    h->phantom = phantom_blocks;
    drop_graphs(h);
    return LBKM_OK;
}

lbkm_status lbkm_autotune(lbkm_t h, int32_t trial_steps, int32_t* chosen)
{
    if (!h || trial_steps < 1) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm_autotune before init");
    if (!h->batched) {
        if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
        return LBKM_OK; // single grids use their fixed plan
    }
    int sms = 0, dev = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    // keep the state and counters; every trial starts from them
    DevTemp saved_t(h);
    CUDA_TRY(h, dmalloc(h, &saved_t.p, h->state_bytes_dev));
    void* saved = saved_t.p;
    DevCounters c0;
    const int cur0 = h->cur;
    const int64_t steps0 = h->host_steps;
    cudaError_t e = cudaMemcpy(saved, h->buf[cur0], h->state_bytes_dev, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(&c0, h->ctr, sizeof(c0), cudaMemcpyDeviceToHost);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    float best = -1.f;
    int best_bt = h->bt, best_grid = h->bgrid;
    const int bts[2] = {64, 128};
    for (int t = 0; t < 2 && e == cudaSuccess; t++) {
        const int maxb = batch_max_blocks(h->recovery, bts[t]);
        for (int bps = 1; bps <= maxb && e == cudaSuccess; bps++) {
            h->bt = bts[t];
            h->bgrid = bps * sms;
            e = build_items(h, batch_segment(h->bt));
            if (e != cudaSuccess) break;
            h->cur = cur0;
            e = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream);
            if (e == cudaSuccess)
                e = launch_batch(h->recovery, h->bt, h->Kf, batch_args(h, 1), h->bgrid, h->stream);
            h->cur = cur0 ^ 1;
            if (e == cudaSuccess) e = cudaEventRecord(ev0, h->stream);
            if (e == cudaSuccess)
                e = launch_batch(h->recovery, h->bt, h->Kf, batch_args(h, trial_steps), h->bgrid,
                                 h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e == cudaSuccess && (best < 0.f || ms < best)) {
                best = ms;
                best_bt = h->bt;
                best_grid = h->bgrid;
            }
            // back to the saved state
            h->cur = cur0;
            if (e == cudaSuccess)
                e = cudaMemcpy(h->buf[cur0], saved, h->state_bytes_dev, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(h->ctr, &c0, sizeof(c0), cudaMemcpyHostToDevice);
        }
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    h->host_steps = steps0;
    h->cur = cur0;
    h->bt = best_bt;
    h->bgrid = best_grid;
    if (e == cudaSuccess) e = build_items(h, batch_segment(h->bt));
    drop_graphs(h);
    if (e != cudaSuccess) return fail(h, LBKM_ECUDA, "autotune: %s", cudaGetErrorString(e));
    lbkm_status st = check_status(h);
    if (st != LBKM_OK) return st;
    if (chosen) {
        chosen[0] = h->bt;
        chosen[1] = h->bgrid / (sms > 0 ? sms : 1);
        chosen[2] = h->bgrid;
    }
    return LBKM_OK;
}

// the conditions lbkm_grad and lbkm_objective_value share
static lbkm_status objective_check(lbkm_t h, const lbkm_objective* ob, const char* fn)
{
    if (h->ny != 1 || h->batched)
        return fail(h, LBKM_EINVAL, "%s needs a single grid with ny = 1", fn);
    if (h->p.bc_x == LBKM_BC_SIDES)
        return fail(h, LBKM_EINVAL, "%s needs periodic or zero-gradient ends", fn);
    if (h->p.bc_x == LBKM_BC_PERIODIC && h->nx < 5)
        return fail(h, LBKM_EINVAL, "%s needs nx >= 5 on a periodic grid", fn);
    if (h->p.time_scheme != 0) return fail(h, LBKM_EINVAL, "%s needs forward Euler", fn);
    if (!h->initialized) return fail(h, LBKM_ESTATE, "%s before lbkm_init_fields", fn);
    if (!ob->rho_target || ob->steps < 1 || ob->checkpoint_every < 1)
        return fail(h, LBKM_EINVAL, "rho_target, steps >= 1 and checkpoint_every >= 1 needed");
    return LBKM_OK;
}

lbkm_status lbkm_grad(lbkm_t h, const lbkm_objective* ob, lbkm_grad_out* out)
{
    if (!h || !ob || !out) return LBKM_EINVAL;
    {
        const lbkm_status cs = objective_check(h, ob, "lbkm_grad");
        if (cs != LBKM_OK) return cs;
    }
    const int nx = h->nx;
    const int64_t N = ob->steps;
    const int C = ob->checkpoint_every;
    const int64_t nck = (N + C - 1) / C;
    const int G = adj_grid(nx);
    // With an FP32 handle the forward run is the FP32 step and keeps FP32 checkpoints;
    // each segment is recomputed in FP64 from its checkpoint widened to FP64 and reversed
    // in FP64, so the derivative is taken along FP64 segments restarted from the FP32
    // run's states. (The exact adjoint of the FP32 step itself is not usable over long
    // runs: on flat stretches FP32 rounding decides the limiter's branches every step,
    // and the limiter's linearisation about such a state amplifies the adjoint.)
    const bool f32 = h->precision != LBKM_F64;
    const size_t SBf = h->state_bytes_dev;                  // forward states, checkpoints
    const size_t SBd = (size_t)NPLANE * h->plane_elems * 8; // FP64 segment states
    char *ck = nullptr, *seg = nullptr;
    double *work = nullptr, *mats = nullptr;
    DevCounters* sctr = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        dfree(h, ck);
        dfree(h, seg);
        dfree(h, work);
        dfree(h, mats);
        dfree(h, sctr);
    };
    // work: mac 4n, mb 16n, loc 6n, gb 2n, fbA/fbB 32n, lbA/lbB 2n, rho_t n, drho0 n,
    //       cw 85n, pacc NPAR*G, jtne G, jmis G
    const size_t nwork = (size_t)nx * (4 + 16 + 6 + 2 + 32 + 2 + 1 + 1 + 85) + (size_t)(ADJ_NPAR + 2) * G;
    cudaError_t e = dmalloc(h, &ck, SBf * nck);
    if (e == cudaSuccess) e = dmalloc(h, &seg, SBd * (size_t)(C + 1));
    if (e == cudaSuccess) e = dmalloc(h, &work, sizeof(double) * nwork);
    if (e == cudaSuccess) e = dmalloc(h, &mats, sizeof(double) * 16);
    if (e == cudaSuccess) e = dmalloc(h, &sctr, sizeof(DevCounters));
    if (e != cudaSuccess) {
        cleanup();
        return fail(h, e == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA,
                    "lbkm_grad allocation: %s", cudaGetErrorString(e));
    }
    double* mac = work;
    double* mb = mac + 4 * (size_t)nx;
    double* loc = mb + 16 * (size_t)nx;
    double* gb = loc + 6 * (size_t)nx;
    double* fbA = gb + 2 * (size_t)nx;
    double* fbB = fbA + 16 * (size_t)nx;
    double* lbA = fbB + 16 * (size_t)nx;
    double* lbB = lbA + nx;
    double* rho_t = lbB + nx;
    double* drho0 = rho_t + nx;
    double* cw = drho0 + nx;
    double* pacc = cw + 85 * (size_t)nx;
    double* jtne = pacc + (size_t)ADJ_NPAR * G;
    double* jmis = jtne + G;
    std::vector<double> hm(16); // x-velocities of the 16 f_i
    {
        static const int ax[4] = {1, 0, -1, 0}, dg[4] = {1, -1, -1, 1};
        for (int o = 0; o < 4; o++)
            for (int q = 0; q < 4; q++)
                hm[4 * o + q] = h->hm.c[o] * (h->p.orbit_kind[o] == 0 ? ax[q] : dg[q]);
    }
    cudaStream_t st = h->stream;
    auto S = [&](int64_t k) { return seg + (size_t)k * SBd; };
    auto K_ = [&](int64_t k) { return ck + (size_t)k * SBf; };
#define GT(call)                                                                              \
    do {                                                                                      \
        e = (call);                                                                           \
        if (e != cudaSuccess) {                                                               \
            cleanup();                                                                        \
            return fail(h, LBKM_ECUDA, "lbkm_grad: %s: %s", #call, cudaGetErrorString(e));   \
        }                                                                                     \
    } while (0)
    GT(cudaMemcpyAsync(mats, hm.data(), sizeof(double) * hm.size(), cudaMemcpyHostToDevice, st));
    GT(cudaMemcpyAsync(rho_t, ob->rho_target, sizeof(double) * nx, cudaMemcpyHostToDevice, st));
    GT(cudaMemsetAsync(pacc, 0, sizeof(double) * (ADJ_NPAR + 2) * G, st));
    GT(cudaMemsetAsync(sctr, 0, sizeof(DevCounters), st));
    GT(cudaMemcpyAsync(K_(0), h->buf[h->cur], SBf, cudaMemcpyDeviceToDevice, st));
    StepLaunch sl = step_args(h, 0);
    sl.ctr = sctr;
    sl.tne_every = 0;
    StepLaunch sd = sl; // the FP64 step of the recomputed segments
    sd.grid = step_grid(0, 0, false, nx, 1, h->Kd.sbc);
    // forward run in the handle's precision, keeping a state every C steps
    for (int64_t n = 0; n < N; n++) {
        sl.in = n == 0 ? (const void*)K_(0) : (const void*)S(n % 2);
        sl.out = S((n + 1) % 2);
        GT(launch_step(h->precision, h->recovery, false, model_ptr(h), sl, st));
        if ((n + 1) % C == 0 && n + 1 < N)
            GT(cudaMemcpyAsync(K_((n + 1) / C), S((n + 1) % 2), SBf, cudaMemcpyDeviceToDevice, st));
    }
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.mac = mac;
    a.mb = mb;
    a.loc = loc;
    a.gb = gb;
    a.cw = cw;
    a.pacc = pacc;
    a.vx = mats;
    a.tne_w = ob->w_tne * h->p.dx * h->p.dt;
    a.jw = a.tne_w;
    // FP64 forward: seed with the mismatch of the final state now; FP32 forward: once the
    // last segment has been recomputed in FP64
    a.fb0 = fbA;
    a.lb0 = lbA;
    auto seed = [&](const void* final_state) -> cudaError_t {
        a.f = static_cast<const double*>(final_state);
        a.jacc = jmis;
        const cudaError_t se = launch_adj_seed(h->Kd, a, rho_t, ob->w_mismatch, G, st);
        a.jacc = jtne;
        return se;
    };
    if (!f32) GT(seed(S(N % 2)));
    double *fc = fbA, *fn = fbB, *lc = lbA, *ln = lbB;
    for (int64_t sg = nck - 1; sg >= 0; sg--) {
        const int64_t n0 = sg * C, n1 = (n0 + C < N) ? n0 + C : N;
        const bool last = f32 && sg == nck - 1; // recompute through the final state
        if (f32)
            GT(launch_adj_widen(reinterpret_cast<const float*>(K_(sg)), reinterpret_cast<double*>(S(0)),
                                (size_t)NPLANE * h->plane_elems, G, st));
        else
            GT(cudaMemcpyAsync(S(0), K_(sg), SBf, cudaMemcpyDeviceToDevice, st));
        for (int64_t n = n0; n < (last ? n1 : n1 - 1); n++) {
            sd.in = S(n - n0);
            sd.out = S(n - n0 + 1);
            GT(launch_step(0, 0, false, &h->Kd, sd, st));
        }
        if (last) GT(seed(S(n1 - n0)));
        for (int64_t n = n1 - 1; n >= n0; n--) {
            const double* state = reinterpret_cast<const double*>(S(n - n0));
            GT(launch_macros(0, h->Kd, state, mac, mac + nx, mac + 2 * (size_t)nx,
                             mac + 3 * (size_t)nx, nullptr, nullptr, st));
            a.f = state;
            a.fb1 = fc;
            a.lb1 = lc;
            a.fb0 = fn;
            a.lb0 = ln;
            GT(launch_adj_step(h->Kd, a, G, st));
            std::swap(fc, fn);
            std::swap(lc, ln);
        }
    }
    // dJ/drho0 at the start: the FP64 state (for an FP32 handle its widening, which the
    // first segment's recomputation left in S(0))
    a.f = reinterpret_cast<const double*>(f32 ? S(0) : K_(0));
    a.fb1 = fc;
    GT(launch_adj_rho0(h->Kd, a, drho0, G, st));
    std::vector<double> hp((size_t)(ADJ_NPAR + 2) * G);
    GT(cudaMemcpyAsync(hp.data(), pacc, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    if (out->drho0)
        GT(cudaMemcpyAsync(out->drho0, drho0, sizeof(double) * nx, cudaMemcpyDeviceToHost, st));
    if (out->df0)
        GT(cudaMemcpyAsync(out->df0, fc, sizeof(double) * 16 * nx, cudaMemcpyDeviceToHost, st));
    GT(cudaStreamSynchronize(st));
#undef GT
    int stat = 0;
    cudaMemcpy(&stat, &sctr->status, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (stat & 1)
        return fail(h, LBKM_EUNSTABLE, "the forward run reached a non-physical state");
    double sums[ADJ_NPAR + 2];
    for (int q = 0; q < ADJ_NPAR + 2; q++) {
        double s = 0.0;
        for (int b = 0; b < G; b++) s += hp[(size_t)q * G + b];
        sums[q] = s;
    }
    for (int k = 0; k < 16; k++) out->dS[k] = k < 4 ? 0.0 : sums[k - 4];
    out->dQ = sums[12];
    out->domega1 = sums[13];
    out->domega2 = sums[14];
    out->J_tne = sums[ADJ_NPAR];
    out->J_mismatch = sums[ADJ_NPAR + 1];
    out->J = out->J_mismatch + out->J_tne;
    return LBKM_OK;
}

lbkm_status lbkm_objective_value(lbkm_t h, const lbkm_objective* ob, double* J,
                                 double* J_mismatch, double* J_tne)
{
    if (!h || !ob || !J) return LBKM_EINVAL;
    {
        const lbkm_status cs = objective_check(h, ob, "lbkm_objective_value");
        if (cs != LBKM_OK) return cs;
    }
    const int nx = h->nx;
    const int64_t N = ob->steps;
    const int C = ob->checkpoint_every;
    const int G = adj_grid(nx);
    // the same J as lbkm_grad: an FP64 handle's own run; for an FP32 handle, FP64 segments
    // of C steps restarted from the FP32 run's state at their start (the FP32 run goes on
    // beside them, so no checkpoint is kept)
    const bool f32 = h->precision != LBKM_F64;
    const size_t SBf = h->state_bytes_dev;
    const size_t SBd = (size_t)NPLANE * h->plane_elems * 8;
    char *run = nullptr, *seg = nullptr;
    double* work = nullptr;
    DevCounters* sctr = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        dfree(h, run);
        dfree(h, seg);
        dfree(h, work);
        dfree(h, sctr);
    };
    // work: fb 16n, lb n (written by the seed kernel), rho_t n, jtne G, jmis G
    const size_t nwork = (size_t)nx * (16 + 1 + 1) + (size_t)2 * G;
    cudaError_t e = dmalloc(h, &run, SBf * 2);
    if (e == cudaSuccess && f32) e = dmalloc(h, &seg, SBd * 2);
    if (e == cudaSuccess) e = dmalloc(h, &work, sizeof(double) * nwork);
    if (e == cudaSuccess) e = dmalloc(h, &sctr, sizeof(DevCounters));
    if (e != cudaSuccess) {
        cleanup();
        return fail(h, e == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA,
                    "lbkm_objective_value allocation: %s", cudaGetErrorString(e));
    }
    double* fb = work;
    double* lb = fb + 16 * (size_t)nx;
    double* rho_t = lb + nx;
    double* jtne = rho_t + nx;
    double* jmis = jtne + G;
    cudaStream_t st = h->stream;
#define GT(call)                                                                              \
    do {                                                                                      \
        e = (call);                                                                           \
        if (e != cudaSuccess) {                                                               \
            cleanup();                                                                        \
            return fail(h, LBKM_ECUDA, "lbkm_objective_value: %s: %s", #call,                \
                        cudaGetErrorString(e));                                               \
        }                                                                                     \
    } while (0)
    GT(cudaMemcpyAsync(rho_t, ob->rho_target, sizeof(double) * nx, cudaMemcpyHostToDevice, st));
    GT(cudaMemsetAsync(jtne, 0, sizeof(double) * 2 * G, st));
    GT(cudaMemsetAsync(sctr, 0, sizeof(DevCounters), st));
    StepLaunch sl = step_args(h, 0);
    sl.ctr = sctr;
    sl.tne_every = 0;
    StepLaunch sd = sl; // the FP64 step of the segments
    sd.grid = step_grid(0, 0, false, nx, 1, h->Kd.sbc);
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    a.fb0 = fb;
    a.lb0 = lb;
    a.jacc = jtne;
    a.jw = ob->w_tne * h->p.dx * h->p.dt;
    // the TNE term of one FP64 state
    auto tne_term = [&](const void* state) -> cudaError_t {
        a.f = static_cast<const double*>(state);
        return launch_adj_jtne(h->Kd, a, G, st);
    };
    // the run in the handle's precision: m steps taken so far, its state in cur
    const void* cur = h->buf[h->cur];
    int64_t m = 0;
    auto advance = [&]() -> cudaError_t {
        sl.in = cur;
        sl.out = run + (size_t)(m % 2) * SBf;
        const cudaError_t se = launch_step(h->precision, h->recovery, false, model_ptr(h), sl, st);
        cur = sl.out;
        m++;
        return se;
    };
    const void* fin = nullptr; // the FP64 state after N steps
    if (!f32) {
        for (int64_t n = 0; n < N; n++) {
            GT(tne_term(cur));
            GT(advance());
        }
        fin = cur;
    } else {
        for (int64_t n0 = 0; n0 < N; n0 += C) {
            const int64_t n1 = (n0 + C < N) ? n0 + C : N;
            const bool last = n1 == N;
            GT(launch_adj_widen(static_cast<const float*>(cur), reinterpret_cast<double*>(seg),
                                (size_t)NPLANE * h->plane_elems, G, st));
            for (int64_t n = n0; n < n1; n++) {
                const int64_t k = n - n0;
                GT(tne_term(seg + (size_t)(k % 2) * SBd));
                if (n + 1 < n1 || last) {
                    sd.in = seg + (size_t)(k % 2) * SBd;
                    sd.out = seg + (size_t)((k + 1) % 2) * SBd;
                    GT(launch_step(0, 0, false, &h->Kd, sd, st));
                }
            }
            if (last)
                fin = seg + (size_t)((n1 - n0) % 2) * SBd;
            else
                for (int64_t n = n0; n < n1; n++) GT(advance());
        }
    }
    a.f = static_cast<const double*>(fin);
    a.jacc = jmis;
    GT(launch_adj_seed(h->Kd, a, rho_t, ob->w_mismatch, G, st));
    std::vector<double> hp((size_t)2 * G);
    GT(cudaMemcpyAsync(hp.data(), jtne, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    GT(cudaStreamSynchronize(st));
#undef GT
    int stat = 0;
    cudaMemcpy(&stat, &sctr->status, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (stat & 1)
        return fail(h, LBKM_EUNSTABLE, "the forward run reached a non-physical state");
    double jt = 0.0, jm = 0.0;
    for (int b = 0; b < G; b++) jt += hp[b];
    for (int b = 0; b < G; b++) jm += hp[(size_t)G + b];
    *J = jm + jt;
    if (J_mismatch) *J_mismatch = jm;
    if (J_tne) *J_tne = jt;
    return LBKM_OK;
}

const char* lbkm_last_error(lbkm_t h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

int32_t lbkm_version(void) { return 100; }

} // extern "C"

namespace lbk {
// Message for lbkm_last_error(NULL) from entry points that take no handle.
void set_handleless_error(const char* msg) { g_create_error = msg; }
} // namespace lbk
