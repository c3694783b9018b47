// lbm_api.cu -- the C-ABI of include/lbm.h: argument checks, workspace layout,
// host <-> device staging, step launches and the autotuner.
//
// Workspace layout (caller-owned, 256-byte aligned):
//   [ buffer 0 | buffer 1 | reduction partials | reduction result | status ]
// Buffers hold Q*C values of the storage type each; the step reads the current
// one and writes the other (pull streaming, Eq. lbe).  Host transfers of fields
// are staged through whichever region is idle.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_trace.h"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

lbm_status cuda_fail(cudaError_t e, const char *what) {
    return fail(LBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define LBM_CUDA(call, what)                               \
    do {                                                   \
        cudaError_t e__ = (call);                          \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

struct LatInfo {
    int D, Q, maxc, kmax;
    double T0;
};

template <class LT>
LatInfo info_of() {
    return LatInfo{LT::D, LT::Q, LT::MAXC, LT::KMAX, LT::T0};
}

bool lattice_info(lbm_lattice lat, LatInfo *out) {
    switch (lat) {
    case LBM_D2Q9: *out = info_of<D2Q9>(); return true;
    case LBM_D3Q15: *out = info_of<D3Q15>(); return true;
    case LBM_D3Q19: *out = info_of<D3Q19>(); return true;
    case LBM_D3Q27: *out = info_of<D3Q27>(); return true;
    case LBM_D3Q39: *out = info_of<D3Q39>(); return true;
    }
    return false;
}

template <class LT>
void fill_table(int *c, double *w) {
    for (int i = 0; i < LT::Q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = vel<LT>(i, a);
        if (w) w[i] = weight<LT>(i);
    }
}

size_t storage_size(lbm_storage st) {
    switch (st) {
    case LBM_STORE_F32: return 4;
    case LBM_STORE_F16: return 2;
    case LBM_STORE_BF16: return 2;
    case LBM_STORE_F64: return 8;
    case LBM_STORE_Q16: return 2;
    case LBM_STORE_F16_REF: return 2;
    case LBM_STORE_BF16_REF: return 2;
    }
    return 0;
}

// Stored planes of C values per buffer: Q distributions, plus D reference-velocity planes.
size_t planes_of(const LatInfo &li, lbm_storage st) {
    return size_t(li.Q) + (has_reference_planes(st) ? size_t(li.D) : 0);
}

const KernelSet *kernels_for(lbm_lattice lat, int K, lbm_storage st) {
    switch (lat) {
    case LBM_D2Q9: return kernels_d2q9(K, st);
    case LBM_D3Q15: return kernels_d3q15(K, st);
    case LBM_D3Q19: return kernels_d3q19(K, st);
    case LBM_D3Q27: return kernels_d3q27(K, st);
    case LBM_D3Q39: return kernels_d3q39(K, st);
    }
    return nullptr;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kPartialBytes = size_t(kReduceBlocks) * 4 * sizeof(double);

// Checks dims for a lattice; returns an empty string when valid.
std::string dims_problem(const LatInfo &li, const int64_t *dims) {
    if (!dims) return "dims is NULL";
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1) return "every dimension must be >= 1";
    if (li.D == 2 && dims[2] != 1) return "a 2-D lattice needs nz == 1";
    for (int a = 0; a < li.D; ++a)
        if (dims[a] < li.maxc) return "every dimension must be >= the largest velocity component";
    if (dims[0] > (1 << 24) || dims[1] > (1 << 24) || dims[2] > 65535) return "dimension too large";
    const double cells = double(dims[0]) * double(dims[1]) * double(dims[2]);
    if (cells > 2147483647.0) return "more than 2^31-1 cells per velocity plane";
    return std::string();
}

}  // namespace

namespace lbm {
// Records a message for lbm_last_error (used by the other C-ABI units).
lbm_status set_error(lbm_status s, const char *msg) { return fail(s, "%s", msg); }
lbm_status set_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

bool lattice_query(lbm_lattice lat, int *D, int *Q, int *maxc, int *kmax) {
    LatInfo li;
    if (!lattice_info(lat, &li)) return false;
    *D = li.D;
    *Q = li.Q;
    *maxc = li.maxc;
    *kmax = li.kmax;
    return true;
}
size_t storage_bytes(lbm_storage st) { return storage_size(st); }
const KernelSet *kernel_set(lbm_lattice lat, int K, lbm_storage st) { return kernels_for(lat, K, st); }
std::string dims_check(lbm_lattice lat, const int64_t *dims) {
    LatInfo li;
    if (!lattice_info(lat, &li)) return "unknown lattice";
    return dims_problem(li, dims);
}
}  // namespace lbm

struct lbm_solver {
    lbm_lattice lat;
    LatInfo li;
    int K;
    lbm_storage st;
    size_t ssize;
    int nx, ny, nz;
    long long C;
    double tau, rho0, relax;
    char *ws;
    size_t ws_bytes, buf_bytes;
    void *buf[2];
    int cur;
    double *partials;
    double *red_out;
    unsigned int *status;
    cudaStream_t stream;
    long long t;
    const KernelSet *ks;       // the kernels the solver runs: ks_base, or its shifted companion
    const KernelSet *ks_base;  // the kernels of its (lattice, K, storage)
    int variant, V, block;
    lbm_collision model;
    double theta;  // energy-flux weight (Eq. pq); 0 = the paper's Sec. 3 collision
    int qexp;      // fixed-point storage: grid step 2^qexp (range 2^(qexp + 15))
    bool qauto;    // fixed-point storage: choose the range at each lbm_set_fields
    bool qref_on;  // fixed-point storage: values stored relative to the equilibrium at qref_u
    double qref_u[3];
    double qref_h[kQMax];  // that equilibrium as scaled shifted values, per velocity
    double graph_theta;
    // Captured graphs of kGraphSteps consecutive steps, one per starting buffer; rebuilt
    // when the kernel configuration changes.  They cut the per-step launch cost, which
    // dominates on small lattices.
    cudaGraphExec_t graph[2];
    int graph_cfg[3];
    cudaStream_t capture;
};

namespace {

// Codec constants of the solver's storage: grid step and reference shift.
QScale solver_qscale(const lbm_solver *s) {
    return qscale_of_exponent(s->qexp, s->qref_on ? s->qref_h : nullptr, s->li.Q);
}

// Smallest grid exponent the reference shift allows: k_i = ref_i / 2^e must stay below 2^22.
int min_qexp_for_reference(const lbm_solver *s) {
    if (!s->qref_on) return -1000;
    double m = 0.0;
    for (int i = 0; i < s->li.Q; ++i) m = std::max(m, fabs(s->qref_h[i]));
    int e = -40;
    while (e < 30 && ldexp(m, -e) >= 4194304.0) ++e;  // 2^22
    return e;
}

StepArgs step_args(const lbm_solver *s, int from) {
    StepArgs a = {};
    a.src = s->buf[from];
    a.dst = s->buf[from ^ 1];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.P = s->C;
    a.relax = s->relax;
    a.rho0 = s->rho0;
    a.status = s->status;
    a.grid_limit = 0;
    a.theta = s->theta;
    a.qs = solver_qscale(s);
    return a;
}

step_fn step_for(const lbm_solver *s, int variant, int V) {
    if (s->model == LBM_COLLISION_BGK) return (variant == 0 && V == 1) ? s->ks->bgk : nullptr;
    if (s->theta != 0.0) return (variant == 0 && V == 1) ? s->ks->theta : nullptr;
    if (variant == 0) {
        int k = v_index(V);
        if (k < 0 || s->nx % V) return nullptr;
        return s->ks->direct[k];
    }
    if (variant == 1)
        return (s->ks->staged && s->ks->staged_applies && s->ks->staged_applies(s->nx)) ? s->ks->staged : nullptr;
    if (variant == 2) return V == 2 ? s->ks->pair : nullptr;  // two cells of the flat index per thread
    return nullptr;
}

lbm_status check_solver(const lbm_solver *s) {
    if (!s) return fail(LBM_ERR_INVALID_ARG, "solver is NULL");
    return LBM_OK;
}

// Staging region for host transfers: the idle distribution buffer, or the
// reduction partials when they are larger (tiny lattices).
void staging(const lbm_solver *s, int busy, char **ptr, size_t *bytes) {
    if (s->buf_bytes >= kPartialBytes) {
        *ptr = static_cast<char *>(s->buf[busy ^ 1]);
        *bytes = s->buf_bytes;
    } else {
        *ptr = reinterpret_cast<char *>(s->partials);
        *bytes = kPartialBytes;
    }
}

// The kernels record events in the workspace's status word (kStatus* bits): a
// bounded-wait expiry of the staged step, a value outside the fixed-point storage's
// range.  The synchronous calls read (and clear) it.
lbm_status check_device_status(lbm_solver *s) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, s->status, sizeof(v), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    if (v != 0) {
        cudaMemsetAsync(s->status, 0, sizeof(unsigned int), s->stream);
        if (v & kStatusBounds)
            return fail(LBM_ERR_BOUNDS, "an index fell outside its buffer (bounds-check build; status 0x%x)", v);
        if (v & kStatusTimeout)
            return fail(LBM_ERR_TIMEOUT, "a bounded wait in the staged step expired (status 0x%x)", v);
        return fail(LBM_ERR_RANGE, "a value left the fixed-point storage range +-2^%d (status 0x%x)", s->qexp + 15, v);
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_status_string(lbm_status st) {
    switch (st) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
    case LBM_ERR_OUT_OF_MEMORY: return "out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NONFINITE: return "non-finite value";
    case LBM_ERR_TIMEOUT: return "timeout";
    case LBM_ERR_BUSY: return "busy";
    case LBM_ERR_NOT_FOUND: return "not found";
    case LBM_ERR_RANGE: return "value outside the storage range";
    case LBM_ERR_BOUNDS: return "index outside its buffer (bounds-check build)";
    }
    return "unknown status";
}

const char *lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_lattice_info(lbm_lattice lat, int *D, int *Q, int *c, double *w, double *T0, int *kmax) {
    LatInfo li;
    if (!lattice_info(lat, &li)) return fail(LBM_ERR_INVALID_ARG, "unknown lattice %d", int(lat));
    if (D) *D = li.D;
    if (Q) *Q = li.Q;
    if (T0) *T0 = li.T0;
    if (kmax) *kmax = li.kmax;
    switch (lat) {
    case LBM_D2Q9: fill_table<D2Q9>(c, w); break;
    case LBM_D3Q15: fill_table<D3Q15>(c, w); break;
    case LBM_D3Q19: fill_table<D3Q19>(c, w); break;
    case LBM_D3Q27: fill_table<D3Q27>(c, w); break;
    case LBM_D3Q39: fill_table<D3Q39>(c, w); break;
    }
    return LBM_OK;
}

size_t lbm_workspace_bytes(lbm_lattice lat, const int64_t dims[3], lbm_storage st) {
    LatInfo li;
    if (!lattice_info(lat, &li) || storage_size(st) == 0) return 0;
    if (!dims_problem(li, dims).empty()) return 0;
    const size_t C = size_t(dims[0]) * size_t(dims[1]) * size_t(dims[2]);
    const size_t buf = align_up(C * planes_of(li, st) * storage_size(st));
    return 2 * buf + align_up(kPartialBytes) + kAlign + kAlign;
}

lbm_status lbm_create(lbm_lattice lat, const int64_t dims[3], double tau, int K, lbm_storage st, double rho0,
                      void *ws, size_t ws_bytes, void *stream, lbm_solver **out) {
    LBM_NVTX_RANGE("lbm_create");
    if (!out) return fail(LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    LatInfo li;
    if (!lattice_info(lat, &li)) return fail(LBM_ERR_INVALID_ARG, "unknown lattice %d", int(lat));
    if (storage_size(st) == 0) return fail(LBM_ERR_UNSUPPORTED, "unknown storage %d", int(st));
    std::string dp = dims_problem(li, dims);
    if (!dp.empty()) return fail(LBM_ERR_INVALID_ARG, "dims: %s", dp.c_str());
    if (!(tau > 0.5) || !isfinite(tau)) return fail(LBM_ERR_INVALID_ARG, "tau must be finite and > 1/2 (got %g)", tau);
    if (!(rho0 > 0.0) || !isfinite(rho0)) return fail(LBM_ERR_INVALID_ARG, "rho0 must be finite and > 0");
    if (K < 2 || K > li.kmax)
        return fail(LBM_ERR_UNSUPPORTED, "truncation order K=%d outside [2, %d] for this lattice (2N-1)", K, li.kmax);
    if (!ws) return fail(LBM_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(LBM_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    const size_t need = lbm_workspace_bytes(lat, dims, st);
    if (ws_bytes < need)
        return fail(LBM_ERR_OUT_OF_MEMORY, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    const KernelSet *ks = kernels_for(lat, K, st);
    if (!ks) return fail(LBM_ERR_UNSUPPORTED, "no kernels built for this lattice/order/storage");

    lbm_solver *s = new lbm_solver();
    s->lat = lat;
    s->li = li;
    s->K = K;
    s->st = st;
    s->ssize = storage_size(st);
    s->nx = int(dims[0]);
    s->ny = int(dims[1]);
    s->nz = int(dims[2]);
    s->C = (long long)dims[0] * dims[1] * dims[2];
    s->tau = tau;
    s->rho0 = rho0;
    s->relax = 1.0 - 1.0 / tau;
    s->ws = static_cast<char *>(ws);
    s->ws_bytes = ws_bytes;
    s->buf_bytes = size_t(s->C) * planes_of(li, st) * s->ssize;
    const size_t bufa = align_up(s->buf_bytes);
    s->buf[0] = s->ws;
    s->buf[1] = s->ws + bufa;
    s->partials = reinterpret_cast<double *>(s->ws + 2 * bufa);
    s->red_out = reinterpret_cast<double *>(s->ws + 2 * bufa + align_up(kPartialBytes));
    s->status = reinterpret_cast<unsigned int *>(s->ws + 2 * bufa + align_up(kPartialBytes) + kAlign);
    s->cur = 0;
    s->stream = static_cast<cudaStream_t>(stream);
    s->t = 0;
    s->ks = ks;
    s->ks_base = ks;
    s->model = LBM_COLLISION_FILTERED_GI;
    s->qexp = -15;  // fixed-point range 1
    s->qauto = false;
    s->qref_on = false;
    s->variant = 0;
    s->block = 256;
    s->V = 1;
    for (int V : {4, 2, 1})
        if (step_for(s, 0, V)) {
            s->V = V;
            break;
        }
    cudaError_t me = cudaMemsetAsync(s->status, 0, sizeof(unsigned int), s->stream);
    if (me != cudaSuccess) {
        delete s;
        return cuda_fail(me, "lbm_create: clear status word");
    }
    *out = s;
    return LBM_OK;
}

static void drop_step_graphs(lbm_solver *s);

lbm_status lbm_destroy(lbm_solver *s) {
    if (!s) return LBM_OK;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    drop_step_graphs(s);
    if (s->capture) cudaStreamDestroy(s->capture);
    delete s;
    if (e != cudaSuccess) return cuda_fail(e, "lbm_destroy: stream synchronize");
    return LBM_OK;
}

// One pass of the init kernel over the whole lattice: f^eq of (rho, u), from device memory
// directly or staged from the host through the idle buffer.
static lbm_status init_pass(lbm_solver *s, const double *rho, const double *u, lbm_mem mem, InitArgs a) {
    const int D = s->li.D;
    if (mem == LBM_MEM_DEVICE) {
        a.rho = rho;
        a.u = u;
        a.ustride = s->C;
        a.c0 = 0;
        a.count = s->C;
        LBM_CUDA(s->ks->init(a, s->stream), "set_fields: init kernel");
        return LBM_OK;
    }
    char *stage;
    size_t cap;
    staging(s, 0, &stage, &cap);
    const long long per = (long long)(cap / (sizeof(double) * (1 + D)));
    if (per < 1) return fail(LBM_ERR_OUT_OF_MEMORY, "staging area too small");
    for (long long c0 = 0; c0 < s->C; c0 += per) {
        const long long n = std::min(per, s->C - c0);
        double *drho = reinterpret_cast<double *>(stage);
        double *du = drho + n;
        LBM_CUDA(cudaMemcpyAsync(drho, rho + c0, n * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                 "set_fields: copy rho");
        for (int d = 0; d < D; ++d)
            LBM_CUDA(cudaMemcpyAsync(du + d * n, u + d * s->C + c0, n * sizeof(double), cudaMemcpyHostToDevice,
                                     s->stream),
                     "set_fields: copy u");
        a.rho = drho;
        a.u = du;
        a.ustride = n;
        a.c0 = c0;
        a.count = n;
        LBM_CUDA(s->ks->init(a, s->stream), "set_fields: init kernel");
    }
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_solver *s, const double *rho, const double *u, lbm_mem mem) {
    LBM_NVTX_RANGE("lbm_set_fields");
    if (lbm_status r = check_solver(s)) return r;
    if (!rho || !u) return fail(LBM_ERR_INVALID_ARG, "rho and u are required");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    InitArgs a = {};
    a.dst = s->buf[0];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.P = s->C;
    a.rho0 = s->rho0;
    a.status = s->status;
    // the state is replaced: events recorded for the old one no longer apply
    LBM_CUDA(cudaMemsetAsync(s->status, 0, sizeof(unsigned int), s->stream), "set_fields: status word");
    a.qs = solver_qscale(s);  // the measuring pass below needs its reference shift
    if (s->st == LBM_STORE_Q16 && s->qauto) {
        // automatic range: measure the largest |h| of f^eq, then take the smallest power of two
        // R >= 1.25 max|h| (headroom for the flow to develop; an exit is still reported)
        unsigned int *hm = reinterpret_cast<unsigned int *>(s->red_out);
        LBM_CUDA(cudaMemsetAsync(hm, 0, sizeof(unsigned int), s->stream), "set_fields: range word");
        InitArgs m = a;
        m.hmax = hm;
        if (lbm_status r = init_pass(s, rho, u, mem, m)) return r;
        unsigned int bits = 0;
        LBM_CUDA(cudaMemcpyAsync(&bits, hm, sizeof(bits), cudaMemcpyDeviceToHost, s->stream), "set_fields: range");
        LBM_CUDA(cudaStreamSynchronize(s->stream), "set_fields: synchronize");
        float h = 0.f;
        memcpy(&h, &bits, sizeof(h));
        if (!isfinite(h)) return fail(LBM_ERR_RANGE, "set_fields: f^eq is not finite");
        int e2 = -8;
        while (e2 < 8 && (ldexp(1.0, e2) < 1.25 * double(h) || e2 - 15 < min_qexp_for_reference(s))) ++e2;
        if (ldexp(1.0, e2) < 1.25 * double(h))
            return fail(LBM_ERR_RANGE, "set_fields: f^eq needs a range above 2^8 (max |h| = %g)", double(h));
        if (e2 - 15 != s->qexp) {
            drop_step_graphs(s);  // the grid step is baked into captured launches
            s->qexp = e2 - 15;
        }
    }
    a.qs = solver_qscale(s);
    if (has_reference_planes(s->st)) {
        // the reference planes first (each cell's own), then the values relative to them
        a.phase = 0;
        if (lbm_status r = init_pass(s, rho, u, mem, a)) return r;
        a.phase = 1;
    }
    if (lbm_status r = init_pass(s, rho, u, mem, a)) return r;
    LBM_CUDA(cudaStreamSynchronize(s->stream), "set_fields: synchronize");
    s->cur = 0;
    s->t = 0;
    return check_device_status(s);  // LBM_ERR_RANGE if f^eq does not fit the fixed-point range
}

static void drop_step_graphs(lbm_solver *s) {
    for (int b = 0; b < 2; ++b)
        if (s->graph[b]) {
            cudaGraphExecDestroy(s->graph[b]);
            s->graph[b] = nullptr;
        }
}

constexpr int kGraphSteps = 32;  // even: a graph leaves the state in the buffer it started from

// Graph of kGraphSteps steps starting from buffer `from` (captured on a private stream).
static cudaError_t step_graph(lbm_solver *s, step_fn fn, int from, cudaGraphExec_t *out) {
    const int cfg2 = s->block + (s->model == LBM_COLLISION_BGK ? 1 << 20 : 0) + (s->theta != 0.0 ? 1 << 21 : 0);
    if (s->theta != s->graph_theta) {  // theta is baked into the captured launches
        drop_step_graphs(s);
        s->graph_theta = s->theta;
    }
    if (s->graph_cfg[0] != s->variant || s->graph_cfg[1] != s->V || s->graph_cfg[2] != cfg2) {
        drop_step_graphs(s);
        s->graph_cfg[0] = s->variant;
        s->graph_cfg[1] = s->V;
        s->graph_cfg[2] = cfg2;
    }
    if (s->graph[from]) {
        *out = s->graph[from];
        return cudaSuccess;
    }
    cudaError_t e = cudaSuccess;
    if (!s->capture) e = cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) le = fn(step_args(s, from ^ (k & 1)), s->block, s->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->capture, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le != cudaSuccess ? le : e;
    }
    e = cudaGraphInstantiate(&s->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph[from] = nullptr;
        return e;
    }
    *out = s->graph[from];
    return cudaSuccess;
}

lbm_status lbm_step(lbm_solver *s, int64_t n) {
    LBM_NVTX_RANGE("lbm_step");
    if (lbm_status r = check_solver(s)) return r;
    if (n < 0) return fail(LBM_ERR_INVALID_ARG, "n must be >= 0");
    step_fn fn = step_for(s, s->variant, s->V);
    if (!fn) return fail(LBM_ERR_UNSUPPORTED, "kernel configuration not built");
    while (n >= kGraphSteps) {
        cudaGraphExec_t g = nullptr;
        cudaError_t e = step_graph(s, fn, s->cur, &g);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: graph capture");
        e = cudaGraphLaunch(g, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: graph launch");
        s->t += kGraphSteps;
        n -= kGraphSteps;
    }
    for (int64_t k = 0; k < n; ++k) {
        StepArgs a = step_args(s, s->cur);
        cudaError_t e = fn(a, s->block, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: launch");
        s->cur ^= 1;
        s->t += 1;
    }
    return LBM_OK;
}

static lbm_status pull_out(lbm_solver *s, double *rho, double *u, double *f, lbm_mem mem) {
    LBM_NVTX_RANGE(f ? "lbm_get_f" : "lbm_get_moments");
    if (lbm_status st = check_device_status(s)) return st;
    const int D = s->li.D, Q = s->li.Q;
    PullArgs a = {};
    a.src = s->buf[s->cur];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.P = s->C;
    a.rho0 = s->rho0;
    a.qs = solver_qscale(s);
    a.status = s->status;
    pull_fn fn = f ? s->ks->pull_f : s->ks->moments;
    if (mem == LBM_MEM_DEVICE) {
        a.rho = rho;
        a.u = u;
        a.f = f;
        a.ustride = s->C;
        a.fstride = s->C;
        a.c0 = 0;
        a.count = s->C;
        LBM_CUDA(fn(a, s->stream), "pull kernel");
    } else {
        char *stage;
        size_t cap;
        staging(s, s->cur, &stage, &cap);
        const int per_cell = f ? Q : ((rho ? 1 : 0) + (u ? D : 0));
        if (per_cell == 0) return LBM_OK;
        const long long per = (long long)(cap / (sizeof(double) * per_cell));
        if (per < 1) return fail(LBM_ERR_OUT_OF_MEMORY, "staging area too small");
        for (long long c0 = 0; c0 < s->C; c0 += per) {
            const long long n = std::min(per, s->C - c0);
            double *base = reinterpret_cast<double *>(stage);
            a.f = f ? base : nullptr;
            a.rho = (!f && rho) ? base : nullptr;
            a.u = (!f && u) ? base + (rho ? n : 0) : nullptr;
            a.ustride = n;
            a.fstride = n;
            a.c0 = c0;
            a.count = n;
            LBM_CUDA(fn(a, s->stream), "pull kernel");
            if (f) {
                for (int i = 0; i < Q; ++i)
                    LBM_CUDA(cudaMemcpyAsync(f + (long long)i * s->C + c0, base + (long long)i * n,
                                             n * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                             "copy f");
            } else {
                if (rho)
                    LBM_CUDA(cudaMemcpyAsync(rho + c0, a.rho, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                             "copy rho");
                if (u)
                    for (int d = 0; d < D; ++d)
                        LBM_CUDA(cudaMemcpyAsync(u + (long long)d * s->C + c0, a.u + (long long)d * n,
                                                 n * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                                 "copy u");
            }
        }
    }
    LBM_CUDA(cudaStreamSynchronize(s->stream), "synchronize");
    if (kBoundsCheck) return check_device_status(s);  // the pull kernel's own accesses
    return LBM_OK;
}

lbm_status lbm_get_moments(lbm_solver *s, double *rho, double *u, lbm_mem mem) {
    if (lbm_status r = check_solver(s)) return r;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    if (!rho && !u) return LBM_OK;
    return pull_out(s, rho, u, nullptr, mem);
}

lbm_status lbm_get_f(lbm_solver *s, double *f, lbm_mem mem) {
    if (lbm_status r = check_solver(s)) return r;
    if (!f) return fail(LBM_ERR_INVALID_ARG, "f is NULL");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    return pull_out(s, nullptr, nullptr, f, mem);
}

static lbm_status reduce_to_host(lbm_solver *s, reduce_fn fn, ReduceArgs &a, int nvals, double *out) {
    LBM_NVTX_RANGE(nvals == 4 ? "lbm_conservation" : "lbm_mode_amplitude");
    if (lbm_status st = check_device_status(s)) return st;
    a.src = s->buf[s->cur];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.P = s->C;
    a.rho0 = s->rho0;
    a.partials = s->partials;
    a.out = s->red_out;
    a.blocks = kReduceBlocks;
    a.qs = solver_qscale(s);
    a.status = s->status;
    LBM_CUDA(fn(a, s->stream), "reduction kernel");
    LBM_CUDA(cudaMemcpyAsync(out, s->red_out, nvals * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
             "copy reduction");
    LBM_CUDA(cudaStreamSynchronize(s->stream), "synchronize");
    if (kBoundsCheck)
        if (lbm_status st = check_device_status(s)) return st;  // the reduction kernel's own accesses
    for (int q = 0; q < nvals; ++q)
        if (!isfinite(out[q])) return fail(LBM_ERR_NONFINITE, "reduction result %d is not finite", q);
    return LBM_OK;
}

lbm_status lbm_conservation(lbm_solver *s, double out[4]) {
    if (lbm_status r = check_solver(s)) return r;
    if (!out) return fail(LBM_ERR_INVALID_ARG, "out is NULL");
    ReduceArgs a = {};
    return reduce_to_host(s, s->ks->conservation, a, 4, out);
}

lbm_status lbm_mode_amplitude(lbm_solver *s, const int64_t k[3], int component, double out[2]) {
    if (lbm_status r = check_solver(s)) return r;
    if (!out || !k) return fail(LBM_ERR_INVALID_ARG, "k and out are required");
    if (component < 0 || component >= s->li.D) return fail(LBM_ERR_INVALID_ARG, "component out of range");
    ReduceArgs a = {};
    const int n[3] = {s->nx, s->ny, s->nz};
    for (int d = 0; d < 3; ++d) {
        long long kk = k[d] % n[d];
        if (kk < 0) kk += n[d];
        a.k[d] = int(kk);
    }
    a.component = component;
    return reduce_to_host(s, s->ks->mode, a, 2, out);
}

lbm_status lbm_get_distributions(lbm_solver *s, void *dst, size_t bytes, lbm_mem mem, int64_t *t) {
    LBM_NVTX_RANGE("lbm_get_distributions");
    if (lbm_status r = check_solver(s)) return r;
    if (!dst) return fail(LBM_ERR_INVALID_ARG, "dst is NULL");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    if (bytes != s->buf_bytes) return fail(LBM_ERR_INVALID_ARG, "bytes must be %zu", s->buf_bytes);
    if (lbm_status st = check_device_status(s)) return st;  // no checkpoint of a state known to be invalid
    LBM_CUDA(cudaMemcpyAsync(dst, s->buf[s->cur], bytes,
                             mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s->stream),
             "get_distributions: copy");
    LBM_CUDA(cudaStreamSynchronize(s->stream), "get_distributions: synchronize");
    if (t) *t = s->t;
    return LBM_OK;
}

lbm_status lbm_set_distributions(lbm_solver *s, const void *src, size_t bytes, lbm_mem mem, int64_t t) {
    LBM_NVTX_RANGE("lbm_set_distributions");
    if (lbm_status r = check_solver(s)) return r;
    if (!src) return fail(LBM_ERR_INVALID_ARG, "src is NULL");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return fail(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    if (bytes != s->buf_bytes) return fail(LBM_ERR_INVALID_ARG, "bytes must be %zu", s->buf_bytes);
    if (t < 0) return fail(LBM_ERR_INVALID_ARG, "t must be >= 0");
    // the state is replaced: events recorded for the old one no longer apply
    LBM_CUDA(cudaMemsetAsync(s->status, 0, sizeof(unsigned int), s->stream), "set_distributions: status word");
    LBM_CUDA(cudaMemcpyAsync(s->buf[0], src, bytes,
                             mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s->stream),
             "set_distributions: copy");
    LBM_CUDA(cudaStreamSynchronize(s->stream), "set_distributions: synchronize");
    s->cur = 0;
    s->t = t;
    return LBM_OK;
}

lbm_status lbm_time(const lbm_solver *s, int64_t *t) {
    if (!s || !t) return fail(LBM_ERR_INVALID_ARG, "solver and t are required");
    *t = s->t;
    return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_solver *s, int variant, int V, int block) {
    if (lbm_status r = check_solver(s)) return r;
    const int nv = variant < 0 ? s->variant : variant;
    const int nV = V ? V : s->V;
    const int nb = block ? block : s->block;
    if (nb < 32 || nb > 1024 || nb % 32) return fail(LBM_ERR_INVALID_ARG, "block_threads must be 32..1024, x32");
    if (v_index(nV) < 0) return fail(LBM_ERR_INVALID_ARG, "cells_per_thread must be 1, 2, 4 or 8");
    if (nv == 0 && s->nx % nV) return fail(LBM_ERR_INVALID_ARG, "cells_per_thread must divide nx");
    if (!step_for(s, nv, nV))
        return fail(LBM_ERR_UNSUPPORTED, "kernel variant %d with %d cells/thread is not built here", nv, nV);
    s->variant = nv;
    s->V = nV;
    s->block = nb;
    return LBM_OK;
}

lbm_status lbm_set_collision(lbm_solver *s, lbm_collision model) {
    if (lbm_status r = check_solver(s)) return r;
    if (model != LBM_COLLISION_FILTERED_GI && model != LBM_COLLISION_BGK)
        return fail(LBM_ERR_INVALID_ARG, "unknown collision model %d", int(model));
    if (model == LBM_COLLISION_BGK && !s->ks->bgk) return fail(LBM_ERR_UNSUPPORTED, "BGK kernel not built");
    s->model = model;
    if (model == LBM_COLLISION_BGK) {
        s->variant = 0;
        s->V = 1;
    } else {
        s->V = 1;
        for (int V : {4, 2, 1})
            if (step_for(s, 0, V)) {
                s->V = V;
                break;
            }
        s->variant = 0;
    }
    return LBM_OK;
}

lbm_status lbm_set_energy_flux(lbm_solver *s, double theta) {
    if (lbm_status r = check_solver(s)) return r;
    if (!isfinite(theta)) return fail(LBM_ERR_INVALID_ARG, "theta must be finite");
    if (theta != 0.0 && s->K < 3)
        return fail(LBM_ERR_UNSUPPORTED, "the energy-flux series starts at Hermite order 3: needs K >= 3");
    if (theta != 0.0 && !s->ks->theta) return fail(LBM_ERR_UNSUPPORTED, "energy-flux kernel not built");
    s->theta = theta;
    s->variant = 0;
    if (theta != 0.0) {
        s->V = 1;
    } else {
        s->V = 1;
        for (int V : {4, 2, 1})
            if (step_for(s, 0, V)) {
                s->V = V;
                break;
            }
    }
    return LBM_OK;
}

lbm_status lbm_set_storage_range(lbm_solver *s, double range) {
    if (lbm_status r = check_solver(s)) return r;
    if (s->st != LBM_STORE_Q16) return fail(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a range");
    if (range == 0.0) {  // automatic: chosen from the fields at each lbm_set_fields
        s->qauto = true;
        return LBM_OK;
    }
    int e2 = 0;
    const double m = frexp(range, &e2);  // range = m 2^e2, m in [1/2, 1)
    if (!(range > 0.0) || !isfinite(range) || m != 0.5 || e2 - 1 < -8 || e2 - 1 > 8)
        return fail(LBM_ERR_INVALID_ARG, "range must be a power of two in [2^-8, 2^8] (got %g)", range);
    const int qexp = (e2 - 1) - 15;
    if (qexp < min_qexp_for_reference(s))
        return fail(LBM_ERR_INVALID_ARG, "range too fine for the reference shift (needs |shift| < 2^22 steps)");
    s->qauto = false;
    if (qexp != s->qexp) {
        drop_step_graphs(s);  // the grid step is baked into captured launches
        s->qexp = qexp;
    }
    return LBM_OK;
}

lbm_status lbm_set_storage_reference(lbm_solver *s, const double U[3]) {
    if (lbm_status r = check_solver(s)) return r;
    if (!U) return fail(LBM_ERR_INVALID_ARG, "U is NULL");
    if (s->st != LBM_STORE_Q16) return fail(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a reference shift");
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(U[a])) return fail(LBM_ERR_INVALID_ARG, "U must be finite");
        if (a < s->li.D) u2 += U[a] * U[a];  // components beyond the lattice's dimension are ignored
    }
    if (u2 > 0.25) return fail(LBM_ERR_INVALID_ARG, "|U| must be <= 1/2");
    int c[kQMax * 3];
    double T0 = 0.0;
    lbm_lattice_info(s->lat, nullptr, nullptr, c, nullptr, &T0, nullptr);
    if (u2 > 0.0 && !s->ks_base->shifted) return fail(LBM_ERR_UNSUPPORTED, "shifted fixed-point kernels not built");
    s->qref_on = u2 > 0.0;
    for (int a = 0; a < 3; ++a) s->qref_u[a] = a < s->li.D ? U[a] : 0.0;
    // (f^eq_i(rho0, U) - w_i rho0) / w_i with the second-order equilibrium: any fixed values
    // serve (the codec adds back exactly what it takes off); these are close to a flow near U
    for (int i = 0; i < s->li.Q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < s->li.D; ++a) cu += c[3 * i + a] * U[a];
        const double sc = cu / T0, v2 = u2 / T0;
        s->qref_h[i] = s->qref_on ? s->rho0 * (sc + 0.5 * (sc * sc - v2)) : 0.0;
    }
    if (!s->qauto && s->qexp < min_qexp_for_reference(s)) s->qexp = min_qexp_for_reference(s);
    s->ks = s->qref_on ? s->ks_base->shifted : s->ks_base;
    drop_step_graphs(s);  // the codec constants and kernels are baked into captured launches
    return LBM_OK;
}

lbm_status lbm_get_storage_range(const lbm_solver *s, double *range) {
    if (!s || !range) return fail(LBM_ERR_INVALID_ARG, "solver and range are required");
    if (s->st != LBM_STORE_Q16) return fail(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a range");
    *range = ldexp(1.0, s->qexp + 15);
    return LBM_OK;
}

lbm_status lbm_get_kernel(const lbm_solver *s, int *variant, int *V, int *block) {
    if (!s) return fail(LBM_ERR_INVALID_ARG, "solver is NULL");
    if (variant) *variant = s->variant;
    if (V) *V = s->V;
    if (block) *block = s->block;
    return LBM_OK;
}

// Autotuner cache (LBM_AUTOTUNE_CACHE=<file>): one line per tuned problem,
//   <key> <variant> <cells_per_thread> <block> <us per step>
// keyed by device name, lattice, K, storage, dims and collision mode.  Lines are appended;
// the last one for a key wins.  A process-wide mutex orders this process's readers and writers.
namespace {
std::mutex g_tune_cache_mu;

std::string tune_key(const lbm_solver *s) {
    cudaDeviceProp prop;
    int dev = 0;
    std::string name = "gpu";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|L%d|K%d|S%d%s|%dx%dx%d|M%d|T%d", name.c_str(), int(s->lat), s->K, int(s->st),
             s->qref_on ? "R" : "", s->nx, s->ny, s->nz, int(s->model), s->theta != 0.0 ? 1 : 0);
    return buf;
}

bool tune_cache_lookup(const char *path, const std::string &key, int *variant, int *V, int *block, double *us) {
    std::lock_guard<std::mutex> lock(g_tune_cache_mu);
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    int v, c, b;
    double t;
    bool found = false;
    while (fscanf(f, "%255s %d %d %d %lf", k, &v, &c, &b, &t) == 5)
        if (key == k) {
            *variant = v;
            *V = c;
            *block = b;
            *us = t;
            found = true;
        }
    fclose(f);
    return found;
}

void tune_cache_store(const char *path, const std::string &key, int variant, int V, int block, double us) {
    std::lock_guard<std::mutex> lock(g_tune_cache_mu);
    FILE *f = fopen(path, "a");
    if (!f) return;  // the cache is an optimisation: a file that cannot be written is skipped
    fprintf(f, "%s %d %d %d %.3f\n", key.c_str(), variant, V, block, us);
    fclose(f);
}
}  // namespace

lbm_status lbm_autotune(lbm_solver *s, int iters, double *best_us) {
    LBM_NVTX_RANGE("lbm_autotune");
    if (lbm_status r = check_solver(s)) return r;
    if (iters < 1) iters = 1;
    const char *cache = getenv("LBM_AUTOTUNE_CACHE");
    const std::string key = cache && *cache ? tune_key(s) : std::string();
    if (!key.empty()) {
        int v = 0, V = 0, b = 0;
        double us = 0.0;
        if (tune_cache_lookup(cache, key, &v, &V, &b, &us) && step_for(s, v, V) && b >= 32 && b <= 1024 &&
            b % 32 == 0) {
            s->variant = v;
            s->V = V;
            s->block = b;
            if (best_us) *best_us = us;
            return LBM_OK;
        }
    }
    cudaEvent_t e0, e1;
    LBM_CUDA(cudaEventCreate(&e0), "autotune: event");
    LBM_CUDA(cudaEventCreate(&e1), "autotune: event");
    float best = 1e30f;
    int bv = s->variant, bV = s->V, bb = s->block;
    StepArgs a = step_args(s, s->cur);  // reads the state, writes only the idle buffer
    struct Cand {
        int variant, V, block;
    };
    Cand cands[16];
    int nc = 0;
    for (int V : {1, 2, 4, 8})
        for (int b : {128, 256})
            if (step_for(s, 0, V) && nc < 16) cands[nc++] = Cand{0, V, b};
    if (step_for(s, 1, 1) && nc < 16) cands[nc++] = Cand{1, 1, s->ks->staged_block};  // where it applies
    for (int b : {128, 256})
        if (step_for(s, 2, 2) && nc < 16) cands[nc++] = Cand{2, 2, b};
    lbm_status rc = LBM_OK;
    for (int k = 0; k < nc && rc == LBM_OK; ++k) {
        step_fn fn = step_for(s, cands[k].variant, cands[k].V);
        if (!fn) continue;  // every candidate was checked above; kept as a guard
        cudaError_t e = cudaSuccess;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = fn(a, cands[k].block, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s->stream);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = fn(a, cands[k].block, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune: candidate launch");
            break;
        }
        if (ms < best) {
            best = ms;
            bv = cands[k].variant;
            bV = cands[k].V;
            bb = cands[k].block;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    s->variant = bv;
    s->V = bV;
    s->block = bb;
    if (best_us) *best_us = 1000.0 * best / iters;
    if (!key.empty()) tune_cache_store(cache, key, bv, bV, bb, 1000.0 * best / iters);
    return LBM_OK;
}

}  // extern "C"
