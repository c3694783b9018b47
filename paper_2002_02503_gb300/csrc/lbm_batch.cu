// lbm_batch.cu -- the pool of include/lbm.h: many independent periodic lattices
// advanced together by the persistent batch kernel, admitted by device memory
// and batched continuously (requests join and leave at chunk boundaries).
//
// Execution model
//   compute stream : per chunk, an H2D copy of the slot table then one graph of
//                    `chunk` steps (step_index 0..chunk-1).  Each step is one launch
//                    of the pool's slot-mode kernel (1, 2 or 4 cells per thread) over
//                    every resident lattice that still has steps left; the launch
//                    boundary is the step's global barrier.
// Every request is stored with its rows padded to a multiple of 4 (pool_pitch), the pad
// cells holding periodic images of the row's first cells, so every request runs the same
// register-pull mode whatever its nx.
//   io stream      : fields upload + f^eq initialisation of new requests, and the
//                    pull of rho, u of finished ones, overlapping the chunks.
// The slot table and its pinned host mirror are double-buffered, so at most two
// chunks are in flight.  Step counts are scheduled on the host: a request's
// parity and remaining steps after each chunk are known without reading back.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "lbm_arena.h"
#include "lbm_internal.h"
#include "lbm_trace.h"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kEventRing = 64;

struct Request {
    int64_t id;
    int nx, ny, nz;
    int px;                            // padded row pitch (pool_pitch(nx))
    long long C;                       // cells nx ny nz
    long long Cp;                      // stored cells per plane px ny nz
    double relax, rho0;
    int64_t steps_total, steps_sched;  // steps launched so far
    int parity;                        // buffer holding the state after the launched steps
    size_t off, bytes;
    void *buf[2];
    unsigned int *status;              // device status word (kStatusRange), after the two buffers
    int qexp;                          // fixed-point storage: this request's grid step 2^qexp
    bool waited_init;                  // compute stream already waits on its init event
    cudaEvent_t init_event;
    long long finish_chunk;            // chunk counter of its last step (-1 while running)
};

}  // namespace

struct lbm_pool {
    lbm_lattice lat;
    int K;
    lbm_storage st;
    int D, Q, maxc;
    size_t ssize;
    const KernelSet *ks;
    Arena arena;
    int max_slots;
    cudaStream_t compute, io, capture;
    int block;
    int grids[3];  // persistent grid of each slot-mode kernel
    int cpt;  // cells per thread of every slot (1, 2 or 4)
    int qexp; // fixed-point storage: grid step 2^qexp
    bool qauto;  // fixed-point storage: each request's range chosen from its own f^eq at admission
    // double-buffered slot tables
    BatchSlot *d_table[2];
    int *d_header[2];
    BatchSlot *h_table[2];
    int *h_header[2];
    std::map<int64_t, Request> reqs;
    std::vector<int64_t> order;       // resident request ids in admission order
    int64_t next_id;
    long long chunks;                 // chunks launched
    long long completed;              // all chunks < completed are known done
    cudaEvent_t chunk_events[kEventRing];
    std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;  // (chunk length, table buffer)
    mutable std::mutex mu;  // every entry point holds it: a pool serialises its own calls
};

namespace {

lbm_status ensure_completed(lbm_pool *p, long long upto_exclusive, bool wait) {
    while (p->completed < upto_exclusive) {
        cudaEvent_t ev = p->chunk_events[p->completed % kEventRing];
        cudaError_t e = wait ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
        if (e == cudaErrorNotReady) return LBM_OK;
        if (e != cudaSuccess) return set_cuda_error(e, "pool: chunk event");
        p->completed += 1;
    }
    return LBM_OK;
}

// A request's arena block: its two distribution buffers (Q planes of Cp = px ny nz stored
// cells), then its status word.
size_t buffer_bytes(int Q, size_t ssize, long long Cp) { return align_up(size_t(Cp) * Q * ssize); }
size_t request_bytes(int Q, size_t ssize, long long Cp) { return 2 * buffer_bytes(Q, ssize, Cp) + kAlign; }

// Reads (and clears) a request's status word on the io stream; LBM_ERR_RANGE if set.
lbm_status request_status(lbm_pool *p, unsigned int *status);

lbm_status get_graph(lbm_pool *p, long long chunk, int b, cudaGraphExec_t *out) {
    auto key = std::make_pair(chunk, b);
    auto it = p->graphs.find(key);
    if (it != p->graphs.end()) {
        *out = it->second;
        return LBM_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: begin capture");
    cudaError_t le = cudaSuccess;
    for (long long s = 0; s < chunk && le == cudaSuccess; ++s)
        le = p->ks->batch(p->d_table[b], p->d_header[b], int(s), p->grids, p->block, p->cpt, p->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->capture, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_cuda_error(le, "pool: capture launch");
    }
    if (e != cudaSuccess) return set_cuda_error(e, "pool: end capture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: instantiate");
    p->graphs[key] = ex;
    *out = ex;
    return LBM_OK;
}

void drop_graphs(lbm_pool *p) {
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
}

lbm_status set_geometry(lbm_pool *p, int block, int cpt) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: device query");
    int grids[3];
    for (int m = 0; m < 3; ++m) {
        const int occ = p->ks->batch_occupancy(block, m);
        if (occ <= 0) return set_error(LBM_ERR_CUDA, "pool: batch kernel occupancy query failed");
        grids[m] = occ * sms;
    }
    p->block = block;
    p->cpt = cpt;
    for (int m = 0; m < 3; ++m) p->grids[m] = grids[m];
    drop_graphs(p);
    return LBM_OK;
}

// Slot mode of the pool: cells per thread 1, 2 or 4 (every request, thanks to the padded pitch).
int slot_mode(const lbm_pool *p, const Request &) { return p->cpt == 4 ? 2 : (p->cpt == 2 ? 1 : 0); }

// Writes the table of resident requests with steps left into buffer b, grouped by slot mode
// (each mode's kernel walks its own unit range); returns the slot count.
int build_table(lbm_pool *p, int b, int *units_total) {
    int n = 0, units = 0;
    for (int m = 0; m < 3; ++m) {
        p->h_header[b][2 + m] = units;
        for (int64_t id : p->order) {
            Request &r = p->reqs[id];
            const int64_t left = r.steps_total - r.steps_sched;
            if (left <= 0 || slot_mode(p, r) != m) continue;
            BatchSlot &s = p->h_table[b][n];
            s.buf[0] = r.buf[0];
            s.buf[1] = r.buf[1];
            s.nx = r.nx;
            s.ny = r.ny;
            s.nz = r.nz;
            s.px = r.px;
            s.mode = m;
            s.ncx = r.px / p->cpt;
            s.threads = int((long long)s.ncx * r.ny * r.nz);
            s.P = r.Cp;
            s.relax = r.relax;
            s.rho0 = r.rho0;
            s.parity = r.parity;
            s.steps_left = int(std::min<int64_t>(left, 1 << 30));
            s.unit0 = units;
            s.units = int((s.threads + p->block - 1) / p->block);
            s.qmul = ldexpf(1.0f, r.qexp);
            s.qinv = ldexpf(1.0f, -r.qexp);
            s.status = r.status;
            fastdiv_init(unsigned(s.ncx), &s.mx, &s.sx);
            fastdiv_init(unsigned(r.ny), &s.my, &s.sy);
            units += s.units;
            ++n;
        }
        p->h_header[b][5 + m] = units;
    }
    p->h_header[b][0] = units;
    p->h_header[b][1] = n;
    *units_total = units;
    return n;
}

lbm_status pull_to(lbm_pool *p, Request &r, double *rho, double *u, lbm_mem mem) {
    const int cur = r.parity;
    PullArgs a = {};
    a.src = r.buf[cur];
    a.nx = r.nx;
    a.ny = r.ny;
    a.nz = r.nz;
    a.px = r.px;
    a.P = r.Cp;
    a.rho0 = r.rho0;
    a.qs = qscale_of_exponent(r.qexp);
    a.f = nullptr;
    a.status = r.status;
    cudaError_t e;
    if (mem == LBM_MEM_DEVICE) {
        a.rho = rho;
        a.u = u;
        a.ustride = r.C;
        a.fstride = r.C;
        a.c0 = 0;
        a.count = r.C;
        e = p->ks->moments(a, p->io);
        if (e != cudaSuccess) return set_cuda_error(e, "pool: moments");
    } else {
        double *stage = static_cast<double *>(r.buf[cur ^ 1]);
        const size_t cap = buffer_bytes(p->Q, p->ssize, r.Cp);
        const int per_cell = (rho ? 1 : 0) + (u ? p->D : 0);
        if (per_cell == 0) return LBM_OK;
        const long long per = (long long)(cap / (sizeof(double) * per_cell));
        for (long long c0 = 0; c0 < r.C; c0 += per) {
            const long long n = std::min(per, r.C - c0);
            a.rho = rho ? stage : nullptr;
            a.u = u ? stage + (rho ? n : 0) : nullptr;
            a.ustride = n;
            a.fstride = n;
            a.c0 = c0;
            a.count = n;
            e = p->ks->moments(a, p->io);
            if (e != cudaSuccess) return set_cuda_error(e, "pool: moments");
            if (rho) {
                e = cudaMemcpyAsync(rho + c0, a.rho, n * sizeof(double), cudaMemcpyDeviceToHost, p->io);
                if (e != cudaSuccess) return set_cuda_error(e, "pool: copy rho");
            }
            if (u)
                for (int d = 0; d < p->D; ++d) {
                    e = cudaMemcpyAsync(u + (long long)d * r.C + c0, a.u + (long long)d * n, n * sizeof(double),
                                        cudaMemcpyDeviceToHost, p->io);
                    if (e != cudaSuccess) return set_cuda_error(e, "pool: copy u");
                }
        }
    }
    e = cudaStreamSynchronize(p->io);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: io synchronize");
    return LBM_OK;
}

lbm_status request_status(lbm_pool *p, unsigned int *status) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, status, sizeof(v), cudaMemcpyDeviceToHost, p->io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: status word");
    if (v & kStatusBounds) {
        cudaMemsetAsync(status, 0, sizeof(unsigned int), p->io);
        return set_error(LBM_ERR_BOUNDS, "pool: an index of this request fell outside its buffer (bounds-check build)");
    }
    if (v & kStatusRange) {
        cudaMemsetAsync(status, 0, sizeof(unsigned int), p->io);
        return set_error(LBM_ERR_RANGE, "pool: a value of this request left the fixed-point storage range");
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_pool_request_bytes(lbm_lattice lat, const int64_t dims[3], lbm_storage st) {
    int D, Q, maxc, kmax;
    if (!lattice_query(lat, &D, &Q, &maxc, &kmax) || storage_bytes(st) == 0) return 0;
    if (has_reference_planes(st)) return 0;  // pools do not run the reference-velocity forms
    if (!dims_check(lat, dims).empty()) return 0;
    const long long Cp = (long long)pool_pitch(int(dims[0])) * dims[1] * dims[2];
    if (Cp > 2147483647LL) return 0;  // the padded plane must stay within int offsets
    return request_bytes(Q, storage_bytes(st), Cp);
}

lbm_status lbm_pool_create(lbm_lattice lat, int K, lbm_storage st, void *arena, size_t arena_bytes, int max_slots,
                           void *compute_stream, void *io_stream, lbm_pool **out) {
    if (!out) return set_error(LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int D, Q, maxc, kmax;
    if (!lattice_query(lat, &D, &Q, &maxc, &kmax)) return set_error(LBM_ERR_INVALID_ARG, "unknown lattice");
    if (storage_bytes(st) == 0) return set_error(LBM_ERR_UNSUPPORTED, "unknown storage");
    if (K < 2 || K > kmax) return set_error(LBM_ERR_UNSUPPORTED, "truncation order outside [2, 2N-1]");
    if (!arena || reinterpret_cast<uintptr_t>(arena) % kAlign)
        return set_error(LBM_ERR_INVALID_ARG, "arena must be non-NULL and 256-byte aligned");
    if (max_slots < 1 || max_slots > 65536) return set_error(LBM_ERR_INVALID_ARG, "max_slots out of range");
    const size_t meta = 2 * align_up(sizeof(BatchSlot) * max_slots) + 2 * kAlign;
    if (arena_bytes < meta + kAlign) return set_error(LBM_ERR_OUT_OF_MEMORY, "arena too small for the slot tables");
    const KernelSet *ks = kernel_set(lat, K, st);
    if (!ks || !ks->batch) return set_error(LBM_ERR_UNSUPPORTED, "no batch kernel built for this class");

    lbm_pool *p = new lbm_pool();
    p->lat = lat;
    p->K = K;
    p->st = st;
    p->qexp = -15;  // fixed-point range 1
    p->qauto = false;
    p->D = D;
    p->Q = Q;
    p->maxc = maxc;
    p->ssize = storage_bytes(st);
    p->ks = ks;
    p->max_slots = max_slots;
    p->compute = static_cast<cudaStream_t>(compute_stream);
    p->io = static_cast<cudaStream_t>(io_stream);
    p->next_id = 1;
    p->chunks = 0;
    p->completed = 0;
    // tables live at the tail of the arena: the pool allocates no device memory itself
    char *base = static_cast<char *>(arena);
    const size_t tab = align_up(sizeof(BatchSlot) * max_slots);
    char *tail = base + (arena_bytes - meta) / kAlign * kAlign;
    p->d_table[0] = reinterpret_cast<BatchSlot *>(tail);
    p->d_table[1] = reinterpret_cast<BatchSlot *>(tail + tab);
    p->d_header[0] = reinterpret_cast<int *>(tail + 2 * tab);
    p->d_header[1] = reinterpret_cast<int *>(tail + 2 * tab + kAlign);
    p->arena.init(base, size_t(tail - base));
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMallocHost(reinterpret_cast<void **>(&p->h_table[b]), sizeof(BatchSlot) * max_slots);
        if (e == cudaSuccess)
            e = cudaMallocHost(reinterpret_cast<void **>(&p->h_header[b]), kBatchHeaderInts * sizeof(int));
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking);
    for (int k = 0; k < kEventRing && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&p->chunk_events[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lbm_pool_destroy(p);
        return set_cuda_error(e, "pool: host setup");
    }
    lbm_status rs = set_geometry(p, 128, 4);
    if (rs != LBM_OK) {
        lbm_pool_destroy(p);
        return rs;
    }
    *out = p;
    return LBM_OK;
}

lbm_status lbm_pool_submit(lbm_pool *p, const int64_t dims[3], double tau, double rho0, const double *rho,
                           const double *u, lbm_mem mem, int64_t steps, int64_t *id) {
    LBM_NVTX_RANGE("lbm_pool_submit");
    if (!p || !dims || !rho || !u || !id) return set_error(LBM_ERR_INVALID_ARG, "pool, dims, rho, u, id required");
    std::lock_guard<std::mutex> lock(p->mu);
    std::string dp = dims_check(p->lat, dims);
    if (!dp.empty()) return set_error(LBM_ERR_INVALID_ARG, dp.c_str());
    if (!(tau > 0.5) || !isfinite(tau)) return set_error(LBM_ERR_INVALID_ARG, "tau must be finite and > 1/2");
    if (!(rho0 > 0.0) || !isfinite(rho0)) return set_error(LBM_ERR_INVALID_ARG, "rho0 must be > 0");
    if (steps < 0) return set_error(LBM_ERR_INVALID_ARG, "steps must be >= 0");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return set_error(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    if ((int)p->reqs.size() >= p->max_slots) return set_error(LBM_ERR_BUSY, "pool: all slots in use");
    Request r;
    r.nx = int(dims[0]);
    r.ny = int(dims[1]);
    r.nz = int(dims[2]);
    r.px = pool_pitch(r.nx);
    r.C = (long long)dims[0] * dims[1] * dims[2];
    r.Cp = (long long)r.px * dims[1] * dims[2];
    if (r.Cp > 2147483647LL)  // thread and in-plane offsets of the batch kernels are ints
        return set_error(LBM_ERR_INVALID_ARG, "rows padded to a multiple of 4 make more than 2^31-1 cells per plane");
    r.relax = 1.0 - 1.0 / tau;
    r.rho0 = rho0;
    r.steps_total = steps;
    r.steps_sched = 0;
    r.parity = 0;
    r.bytes = request_bytes(p->Q, p->ssize, r.Cp);
    if (!p->arena.alloc(r.bytes, &r.off)) return set_error(LBM_ERR_BUSY, "pool: arena has no room for this request");
    const size_t half = buffer_bytes(p->Q, p->ssize, r.Cp);
    r.buf[0] = p->arena.base + r.off;
    r.buf[1] = p->arena.base + r.off + half;
    r.status = reinterpret_cast<unsigned int *>(p->arena.base + r.off + 2 * half);
    r.waited_init = false;
    r.finish_chunk = steps == 0 ? p->chunks - 1 : -1;
    cudaError_t e = cudaEventCreateWithFlags(&r.init_event, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        p->arena.release(r.off, r.bytes);
        return set_cuda_error(e, "pool: event");
    }
    e = cudaMemsetAsync(r.status, 0, sizeof(unsigned int), p->io);
    if (e != cudaSuccess) {
        cudaEventDestroy(r.init_event);
        p->arena.release(r.off, r.bytes);
        return set_cuda_error(e, "pool: clear status word");
    }
    InitArgs a = {};
    a.dst = r.buf[0];
    a.nx = r.nx;
    a.ny = r.ny;
    a.nz = r.nz;
    a.px = r.px;
    a.P = r.Cp;
    a.rho0 = rho0;
    a.status = r.status;
    // one pass of the init kernel, from device memory or staged through the idle buffer
    auto init_pass = [&](const InitArgs &args) -> cudaError_t {
        InitArgs b = args;
        if (mem == LBM_MEM_DEVICE) {
            b.rho = rho;
            b.u = u;
            b.ustride = r.C;
            b.c0 = 0;
            b.count = r.C;
            return p->ks->init(b, p->io);
        }
        cudaError_t err = cudaSuccess;
        double *stage = static_cast<double *>(r.buf[1]);
        const long long per = (long long)(half / (sizeof(double) * (1 + p->D)));
        for (long long c0 = 0; c0 < r.C && err == cudaSuccess; c0 += per) {
            const long long n = std::min(per, r.C - c0);
            err = cudaMemcpyAsync(stage, rho + c0, n * sizeof(double), cudaMemcpyHostToDevice, p->io);
            for (int d = 0; d < p->D && err == cudaSuccess; ++d)
                err = cudaMemcpyAsync(stage + (1 + d) * n, u + (long long)d * r.C + c0, n * sizeof(double),
                                      cudaMemcpyHostToDevice, p->io);
            b.rho = stage;
            b.u = stage + n;
            b.ustride = n;
            b.c0 = c0;
            b.count = n;
            if (err == cudaSuccess) err = p->ks->init(b, p->io);
        }
        return err;
    };
    r.qexp = p->qexp;
    if (p->st == LBM_STORE_Q16 && p->qauto) {
        // this request's range: the smallest power of two >= 1.25 max|h| of its f^eq, measured
        // into the second word of its status block
        unsigned int *hm = r.status + 1;
        e = cudaMemsetAsync(hm, 0, sizeof(unsigned int), p->io);
        InitArgs m = a;
        m.hmax = hm;
        if (e == cudaSuccess) e = init_pass(m);
        unsigned int bits = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, hm, sizeof(bits), cudaMemcpyDeviceToHost, p->io);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);
        if (e != cudaSuccess) {
            cudaEventDestroy(r.init_event);
            p->arena.release(r.off, r.bytes);
            return set_cuda_error(e, "pool: range measurement");
        }
        float h = 0.f;
        memcpy(&h, &bits, sizeof(h));
        int e2 = -8;
        while (e2 < 8 && ldexp(1.0, e2) < 1.25 * double(h)) ++e2;
        if (!isfinite(h) || ldexp(1.0, e2) < 1.25 * double(h)) {
            cudaEventDestroy(r.init_event);
            p->arena.release(r.off, r.bytes);
            return set_error(LBM_ERR_RANGE, "pool: f^eq does not fit any fixed-point range up to 2^8");
        }
        r.qexp = e2 - 15;
    }
    a.qs = qscale_of_exponent(r.qexp);
    e = init_pass(a);
    if (e == cudaSuccess) e = cudaEventRecord(r.init_event, p->io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);  // host inputs consumed before returning
    if (e != cudaSuccess) {
        cudaEventDestroy(r.init_event);
        p->arena.release(r.off, r.bytes);
        return set_cuda_error(e, "pool: upload");
    }
    if (lbm_status rs = request_status(p, r.status)) {  // f^eq does not fit the fixed-point range
        cudaEventDestroy(r.init_event);
        p->arena.release(r.off, r.bytes);
        return rs;
    }
    r.id = p->next_id++;
    p->reqs[r.id] = r;
    p->order.push_back(r.id);
    *id = r.id;
    return LBM_OK;
}

lbm_status lbm_pool_advance(lbm_pool *p, int64_t chunk, int *active) {
    LBM_NVTX_RANGE("lbm_pool_advance");
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    if (chunk < 1 || chunk > 100000) return set_error(LBM_ERR_INVALID_ARG, "chunk_steps out of range");
    std::lock_guard<std::mutex> lock(p->mu);
    if (active) *active = 0;
    const int b = int(p->chunks & 1);
    // table buffer b was last used by chunk (chunks - 2): wait until every chunk before
    // (chunks - 1) has completed (this also keeps the event ring from overrunning)
    lbm_status rs = ensure_completed(p, p->chunks - 1, true);
    if (rs != LBM_OK) return rs;
    int units = 0;
    const int n = build_table(p, b, &units);
    if (n == 0) return LBM_OK;
    cudaError_t e = cudaSuccess;
    for (int64_t id : p->order) {
        Request &r = p->reqs[id];
        if (!r.waited_init && r.steps_total > r.steps_sched) {
            e = cudaStreamWaitEvent(p->compute, r.init_event, 0);
            if (e != cudaSuccess) return set_cuda_error(e, "pool: wait init");
            r.waited_init = true;
        }
    }
    e = cudaMemcpyAsync(p->d_table[b], p->h_table[b], sizeof(BatchSlot) * n, cudaMemcpyHostToDevice, p->compute);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_header[b], p->h_header[b], kBatchHeaderInts * sizeof(int),
                            cudaMemcpyHostToDevice, p->compute);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: table upload");
    cudaGraphExec_t g;
    rs = get_graph(p, chunk, b, &g);
    if (rs != LBM_OK) return rs;
    e = cudaGraphLaunch(g, p->compute);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: graph launch");
    e = cudaEventRecord(p->chunk_events[p->chunks % kEventRing], p->compute);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: chunk event");
    for (int64_t id : p->order) {
        Request &r = p->reqs[id];
        const int64_t left = r.steps_total - r.steps_sched;
        if (left <= 0) continue;
        const int64_t done = std::min<int64_t>(left, chunk);
        r.steps_sched += done;
        r.parity ^= int(done & 1);
        if (r.steps_sched == r.steps_total) r.finish_chunk = p->chunks;
    }
    p->chunks += 1;
    if (active) *active = n;
    return LBM_OK;
}

lbm_status lbm_pool_poll(lbm_pool *p, int64_t id, int *done, int64_t *steps_done) {
    if (!p || !done) return set_error(LBM_ERR_INVALID_ARG, "pool and done are required");
    std::lock_guard<std::mutex> lock(p->mu);
    auto it = p->reqs.find(id);
    if (it == p->reqs.end()) return set_error(LBM_ERR_NOT_FOUND, "unknown request id");
    lbm_status rs = ensure_completed(p, p->chunks, false);
    if (rs != LBM_OK) return rs;
    const Request &r = it->second;
    *done = (r.finish_chunk >= -1 && r.steps_sched == r.steps_total && r.finish_chunk < p->completed) ? 1 : 0;
    if (steps_done) *steps_done = *done ? r.steps_total : r.steps_sched;
    return LBM_OK;
}

lbm_status lbm_pool_result(lbm_pool *p, int64_t id, double *rho, double *u, lbm_mem mem) {
    LBM_NVTX_RANGE("lbm_pool_result");
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) return set_error(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    std::lock_guard<std::mutex> lock(p->mu);
    auto it = p->reqs.find(id);
    if (it == p->reqs.end()) return set_error(LBM_ERR_NOT_FOUND, "unknown request id");
    Request &r = it->second;
    if (r.steps_sched != r.steps_total) return set_error(LBM_ERR_BUSY, "request has steps left");
    cudaError_t e = cudaStreamWaitEvent(p->io, r.init_event, 0);
    if (e == cudaSuccess && r.finish_chunk >= 0)
        e = cudaStreamWaitEvent(p->io, p->chunk_events[r.finish_chunk % kEventRing], 0);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: order result");
    if (r.finish_chunk >= 0 && r.finish_chunk + kEventRing <= p->chunks) {
        // its chunk event was reused by a later chunk; later completion implies this one
        lbm_status rs = ensure_completed(p, r.finish_chunk + 1, true);
        if (rs != LBM_OK) return rs;
    }
    lbm_status rs = pull_to(p, r, rho, u, mem);
    if (rs != LBM_OK) return rs;
    const lbm_status st = request_status(p, r.status);  // LBM_ERR_RANGE: the outputs are not valid
    cudaEventDestroy(r.init_event);
    p->arena.release(r.off, r.bytes);
    p->order.erase(std::find(p->order.begin(), p->order.end(), id));
    p->reqs.erase(it);
    return st;
}

lbm_status lbm_pool_cancel(lbm_pool *p, int64_t id) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    LBM_NVTX_RANGE("lbm_pool_cancel");
    std::lock_guard<std::mutex> lock(p->mu);
    auto it = p->reqs.find(id);
    if (it == p->reqs.end()) return set_error(LBM_ERR_NOT_FOUND, "unknown request id");
    Request &r = it->second;
    // the launched chunks may still step it, and its upload may still be writing: let both finish
    lbm_status rs = ensure_completed(p, p->chunks, true);
    if (rs != LBM_OK) return rs;
    cudaError_t e = cudaEventSynchronize(r.init_event);
    if (e != cudaSuccess) return set_cuda_error(e, "pool: cancel");
    cudaEventDestroy(r.init_event);
    p->arena.release(r.off, r.bytes);
    p->order.erase(std::find(p->order.begin(), p->order.end(), id));
    p->reqs.erase(it);
    return LBM_OK;
}

lbm_status lbm_pool_sync(lbm_pool *p) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    std::lock_guard<std::mutex> lock(p->mu);
    return ensure_completed(p, p->chunks, true);
}

lbm_status lbm_pool_stats(const lbm_pool *p, size_t *free_bytes, int *resident, int *done) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    std::lock_guard<std::mutex> lock(p->mu);
    if (free_bytes) *free_bytes = p->arena.free_bytes();
    int res = 0, dn = 0;
    for (auto &kv : p->reqs) {
        ++res;
        if (kv.second.steps_sched == kv.second.steps_total && kv.second.finish_chunk < p->completed) ++dn;
    }
    if (resident) *resident = res;
    if (done) *done = dn;
    return LBM_OK;
}

lbm_status lbm_pool_autotune(lbm_pool *p, int iters, double *best_us) {
    LBM_NVTX_RANGE("lbm_pool_autotune");
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    if (iters < 1) iters = 1;
    std::lock_guard<std::mutex> lock(p->mu);
    lbm_status rs = ensure_completed(p, p->chunks, true);
    if (rs != LBM_OK) return rs;
    const int b = int(p->chunks & 1);
    int units = 0;
    // step_index 0 with steps_left >= 1: every launch re-reads the current state and rewrites the idle
    // buffer, so the state is unchanged
    const int n = build_table(p, b, &units);
    if (n == 0) return set_error(LBM_ERR_INVALID_ARG, "pool: no resident request to tune on");
    cudaError_t e = cudaMemcpyAsync(p->d_table[b], p->h_table[b], sizeof(BatchSlot) * n, cudaMemcpyHostToDevice,
                                    p->compute);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_header[b], p->h_header[b], kBatchHeaderInts * sizeof(int),
                            cudaMemcpyHostToDevice, p->compute);
    for (int64_t id : p->order) {
        Request &r = p->reqs[id];
        if (!r.waited_init && e == cudaSuccess) e = cudaStreamWaitEvent(p->compute, r.init_event, 0);
    }
    if (e != cudaSuccess) return set_cuda_error(e, "pool: autotune setup");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_block = p->block, best_cpt = p->cpt;
    for (int cfg = 0; cfg < 6; ++cfg) {
        const int cpt = 1 << (cfg >> 1), block = (cfg & 1) ? 256 : 128;
        rs = set_geometry(p, block, cpt);
        if (rs != LBM_OK) break;
        build_table(p, b, &units);  // units depend on the block size and the cells per thread
        e = cudaMemcpyAsync(p->d_table[b], p->h_table[b], sizeof(BatchSlot) * n, cudaMemcpyHostToDevice, p->compute);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_header[b], p->h_header[b], kBatchHeaderInts * sizeof(int),
                            cudaMemcpyHostToDevice, p->compute);
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            e = p->ks->batch(p->d_table[b], p->d_header[b], 0, p->grids, p->block, p->cpt, p->compute);
        if (e == cudaSuccess) e = cudaEventRecord(e0, p->compute);
        for (int it = 0; it < iters && e == cudaSuccess; ++it)
            e = p->ks->batch(p->d_table[b], p->d_header[b], 0, p->grids, p->block, p->cpt, p->compute);
        if (e == cudaSuccess) e = cudaEventRecord(e1, p->compute);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rs = set_cuda_error(e, "pool: autotune launch");
            break;
        }
        if (ms < best) {
            best = ms;
            best_block = block;
            best_cpt = cpt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != LBM_OK) return rs;
    rs = set_geometry(p, best_block, best_cpt);
    if (rs != LBM_OK) return rs;
    if (best_us) *best_us = 1000.0 * best / iters;
    return LBM_OK;
}

lbm_status lbm_pool_set_storage_range(lbm_pool *p, double range) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->st != LBM_STORE_Q16) return set_error(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a range");
    if (!p->reqs.empty()) return set_error(LBM_ERR_BUSY, "pool: the range can change only while no request is resident");
    if (range == 0.0) {  // automatic: each request's own range, chosen at admission
        p->qauto = true;
        return LBM_OK;
    }
    int e2 = 0;
    const double m = frexp(range, &e2);  // range = m 2^e2, m in [1/2, 1)
    if (!(range > 0.0) || !isfinite(range) || m != 0.5 || e2 - 1 < -8 || e2 - 1 > 8)
        return set_error(LBM_ERR_INVALID_ARG, "range must be a power of two in [2^-8, 2^8], or 0");
    p->qexp = (e2 - 1) - 15;
    p->qauto = false;
    return LBM_OK;
}

lbm_status lbm_pool_get_storage_range(const lbm_pool *p, double *range) {
    if (!p || !range) return set_error(LBM_ERR_INVALID_ARG, "pool and range are required");
    if (p->st != LBM_STORE_Q16) return set_error(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a range");
    std::lock_guard<std::mutex> lock(p->mu);
    *range = p->qauto ? 0.0 : ldexp(1.0, p->qexp + 15);
    return LBM_OK;
}

lbm_status lbm_pool_request_range(const lbm_pool *p, int64_t id, double *range) {
    if (!p || !range) return set_error(LBM_ERR_INVALID_ARG, "pool and range are required");
    if (p->st != LBM_STORE_Q16) return set_error(LBM_ERR_UNSUPPORTED, "only the fixed-point storage has a range");
    std::lock_guard<std::mutex> lock(p->mu);
    auto it = p->reqs.find(id);
    if (it == p->reqs.end()) return set_error(LBM_ERR_NOT_FOUND, "unknown request id");
    *range = ldexp(1.0, it->second.qexp + 15);
    return LBM_OK;
}

lbm_status lbm_pool_set_kernel(lbm_pool *p, int cells_per_thread, int block_threads) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    std::lock_guard<std::mutex> lock(p->mu);
    const int cpt = cells_per_thread == 0 ? p->cpt : cells_per_thread;
    const int block = block_threads == 0 ? p->block : block_threads;
    if (cpt != 1 && cpt != 2 && cpt != 4)
        return set_error(LBM_ERR_UNSUPPORTED, "pool: cells_per_thread must be 1, 2 or 4");
    if (block != 128 && block != 256) return set_error(LBM_ERR_UNSUPPORTED, "pool: block_threads must be 128 or 256");
    // the launched chunks hold graphs built for the current geometry: let them finish first
    lbm_status rs = ensure_completed(p, p->chunks, true);
    if (rs != LBM_OK) return rs;
    return set_geometry(p, block, cpt);
}

lbm_status lbm_pool_get_kernel(const lbm_pool *p, int *cells_per_thread, int *block_threads) {
    if (!p) return set_error(LBM_ERR_INVALID_ARG, "pool is NULL");
    std::lock_guard<std::mutex> lock(p->mu);
    if (cells_per_thread) *cells_per_thread = p->cpt;
    if (block_threads) *block_threads = p->block;
    return LBM_OK;
}

lbm_status lbm_pool_destroy(lbm_pool *p) {
    if (!p) return LBM_OK;
    cudaStreamSynchronize(p->compute);
    cudaStreamSynchronize(p->io);
    drop_graphs(p);
    for (auto &kv : p->reqs) cudaEventDestroy(kv.second.init_event);
    for (int k = 0; k < kEventRing; ++k)
        if (p->chunk_events[k]) cudaEventDestroy(p->chunk_events[k]);
    for (int b = 0; b < 2; ++b) {
        if (p->h_table[b]) cudaFreeHost(p->h_table[b]);
        if (p->h_header[b]) cudaFreeHost(p->h_header[b]);
    }
    if (p->capture) cudaStreamDestroy(p->capture);
    delete p;
    return LBM_OK;
}

}  // extern "C"
