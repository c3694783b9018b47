// lbm_internal.h -- host-side interfaces between the C-ABI layer and the
// per-lattice kernel instantiation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include <string>

#include "../../include/lbm.h"

namespace lbm {

// Cells per thread variants of the register-pull step: V = 1, 2, 4, 8.
constexpr int kNumV = 4;
inline int v_index(int V) { return V == 1 ? 0 : V == 2 ? 1 : V == 4 ? 2 : V == 8 ? 3 : -1; }
inline int v_of_index(int k) { return 1 << k; }

constexpr int kQMax = 39;  // largest velocity count of the built lattices

// Storage forms that keep a per-cell reference velocity in D planes after the Q distribution
// planes (LBM_STORE_F16_REF, LBM_STORE_BF16_REF).
inline bool has_reference_planes(lbm_storage st) { return st == LBM_STORE_F16_REF || st == LBM_STORE_BF16_REF; }

// Constants of the fixed-point storage codec (LBM_STORE_Q16); the floating forms ignore them.
// Grid step 2^e: mul = 2^e, inv = 2^-e.  Per velocity i, a reference shift of k_i whole grid
// steps (k_i = rint(ref_i / 2^e), ref_i the scaled equilibrium at a reference velocity, 0 by
// default) enters the codec's two FMA constants: enc[i] = 2^23 + 2^15 - k_i and
// dec[i] = -(2^23 + 2^15 - k_i) 2^e, both exact in FP32 for |k_i| < 2^22 and |e| <= 30.
// ref[i] keeps the unrounded shift for the range measurement of lbm_set_fields.
struct QScale {
    float mul, inv, off;  // off = -(2^23 + 2^15) 2^e: the decode constant with no shift
    float enc[kQMax], dec[kQMax], ref[kQMax];
};
inline QScale qscale_of_exponent(int e, const double *ref = nullptr, int Q = 0) {
    QScale q;
    q.mul = ldexpf(1.0f, e);
    q.inv = ldexpf(1.0f, -e);
    q.off = -ldexpf(8421376.0f, e);
    for (int i = 0; i < kQMax; ++i) {
        const double k = (ref && i < Q) ? rint(ldexp(ref[i], -e)) : 0.0;
        q.enc[i] = float(8421376.0 - k);
        q.dec[i] = -ldexpf(float(8421376.0 - k), e);
        q.ref[i] = (ref && i < Q) ? float(ref[i]) : 0.0f;
    }
    return q;
}

// Bits of the device status word.
constexpr unsigned int kStatusTimeout = 1u;  // a bounded wait of the staged step expired
constexpr unsigned int kStatusRange = 2u;    // a value left the fixed-point storage's range
constexpr unsigned int kStatusBounds = 4u;   // bounds-check build: an index fell outside its buffer

// The bounds-check build (compiled with -DLBM_DEBUG_BOUNDS, a separate library): every kernel
// checks each computed load and store index against the extent of the buffer (or velocity
// plane) it addresses; an index outside is recorded in the status word and the access is
// skipped -- no trap, the context stays usable -- and the next synchronising call returns
// LBM_ERR_BOUNDS.  In the normal build the checks compile away.
#ifdef LBM_DEBUG_BOUNDS
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

// True when the n elements [first, first + n) lie inside [0, extent).
__host__ __device__ inline bool span_in(long long first, long long n, long long extent) {
    return first >= 0 && n >= 0 && first <= extent - n;
}

#ifdef __CUDACC__
// Bounds-check build: true when the n elements [first, first + n) lie inside [0, extent);
// otherwise records kStatusBounds in *status (when given) and returns false, and the caller
// skips the access.  Constant true in the normal build.
__device__ __forceinline__ bool guard(long long first, int n, long long extent, unsigned int *status) {
    if constexpr (!kBoundsCheck) {
        return true;
    } else {
        if (span_in(first, n, extent)) return true;
        if (status) atomicOr(status, kStatusBounds);
        return false;
    }
}
#endif

struct StepArgs {
    const void *src;  // stored distributions at t (post-collision of t-1, un-streamed)
    void *dst;        // stored distributions at t+1
    int nx, ny, nz;
    long long P;      // cells per velocity plane (nx*ny*nz)
    double relax;     // 1 - 1/tau
    double rho0;
    unsigned int *status;  // device status word (kStatus* bits); may be null for floating storage
    int grid_limit;        // persistent variant: CTAs to launch (0 = one per SM slot)
    double theta;          // weight of the energy-flux part (Eq. pq); 0 = off
    QScale qs;         // fixed-point grid step (LBM_STORE_Q16 only)
};

struct InitArgs {
    void *dst;             // distributions to write
    const double *rho;     // [count] density for cells [c0, c0+count)
    const double *u;       // [D][ustride] velocity (component a at u + a*ustride)
    long long ustride;
    long long c0, count;
    int nx, ny, nz;
    long long P;
    double rho0;
    QScale qs;
    unsigned int *status;  // receives kStatusRange when a value does not fit the fixed-point range
    unsigned int *hmax;    // when set: store nothing, only raise *hmax to the largest |h| (float bits)
    int phase;             // forms with a reference velocity: 0 writes each cell's reference planes,
                           // 1 the distributions relative to the references phase 0 wrote
    int px;                // row pitch of the stored field (0 = nx); pools pad rows to a multiple of 4
                           // and the pad cells x = nx + k hold images of cells k
};

struct PullArgs {
    const void *src;       // stored distributions
    double *rho;           // [count] or null
    double *u;             // [D][ustride] or null
    double *f;             // [Q][fstride] or null (pull_f)
    long long ustride, fstride;
    long long c0, count;
    int nx, ny, nz;
    long long P;
    double rho0;
    QScale qs;
    unsigned int *status;  // bounds-check build: receives kStatusBounds
    int px;                // row pitch of the stored field (0 = nx)
};

struct ReduceArgs {
    const void *src;
    int nx, ny, nz;
    long long P;
    double rho0;
    double *partials;      // [blocks][nvals]
    double *out;           // [nvals] device
    int blocks;
    int k[3];              // mode wave vector
    int component;         // mode velocity component
    QScale qs;
    unsigned int *status;  // bounds-check build: receives kStatusBounds
};

// One lattice of a batch (device-resident table entry).
struct BatchSlot {
    void *buf[2];      // the two distribution buffers of this lattice
    int nx, ny, nz;
    int px;            // row pitch: nx rounded up to a multiple of 4; pad cells hold periodic images
    int mode;          // cells per thread: 0: one, 1: two x-neighbours, 2: four x-neighbours (row vectors)
    int ncx;           // px / V
    int threads;       // threads the slot's step needs (ncx ny nz)
    long long P;       // stored cells per velocity plane (px ny nz)
    double relax;      // 1 - 1/tau
    double rho0;
    int parity;        // buffer holding the state at the start of the chunk
    int steps_left;    // steps still to run at the start of the chunk
    int unit0;         // first work unit of this slot (table sorted by unit0)
    int units;         // work units of this slot
    unsigned int mx, sx, my, sy;  // division by ncx and by ny (fastdiv_init)
    float qmul, qinv;             // fixed-point grid step 2^e and 2^-e (LBM_STORE_Q16 only; no reference shift)
    unsigned int *status;         // this request's status word (kStatusRange)
};

// Header of a slot table: total units, slots, first unit of slot modes 0..2, end unit of
// slot modes 0..2.
constexpr int kBatchHeaderInts = 8;

// Row pitch of a pool request: nx rounded up to a multiple of 4, so that every request can run
// the register pull with up to four cells per thread on aligned row vectors.
inline int pool_pitch(int nx) { return (nx + 3) / 4 * 4; }

// Division by a runtime constant d (1 <= d < 2^31) as q = (umulhi(n, m) + n) >> s for
// 0 <= n < 2^31 -- the round-up multiply-and-shift method of Granlund and Montgomery (1994):
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, so that (m + 2^32) / 2^(32+s) exceeds 1/d by
// less than 2^-(32+s), which keeps n (m + 2^32) / 2^(32+s) below floor(n/d) + 1 for n < 2^31.
inline void fastdiv_init(unsigned int d, unsigned int *m, unsigned int *s) {
    unsigned int l = 0;
    while ((1ull << l) < d) ++l;
    *m = (unsigned int)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    *s = l;
}

typedef cudaError_t (*step_fn)(const StepArgs &, int block_threads, cudaStream_t);
// One step of every slot of the pool's slot mode (cells per thread 1, 2 or 4).
typedef cudaError_t (*batch_fn)(const BatchSlot *slots, const int *header, int step_index, const int *grids,
                                int block, int cells_per_thread, cudaStream_t);
typedef cudaError_t (*init_fn)(const InitArgs &, cudaStream_t);
typedef cudaError_t (*pull_fn)(const PullArgs &, cudaStream_t);
typedef cudaError_t (*reduce_fn)(const ReduceArgs &, cudaStream_t);

struct KernelSet {
    step_fn direct[kNumV];   // variant 0, per V (null where not built)
    step_fn staged;          // variant 1 (null where not built: FP64 and fixed-point storage)
    int staged_block;        // threads per CTA the staged variant is built for
    init_fn init;
    pull_fn moments;
    pull_fn pull_f;
    reduce_fn conservation;  // nvals = 4
    reduce_fn mode;          // nvals = 2
    batch_fn batch;          // persistent multi-lattice step (1, 2 or 4 cells per thread)
    int (*batch_occupancy)(int block, int mode);  // blocks per SM of the slot-mode kernel
    step_fn bgk;             // BGK comparison operator, register pull with V = 1
    step_fn theta;           // filtered collision with the energy-flux term (K >= 3), V = 1
    bool (*staged_applies)(int nx);  // variant 1 needs nx * sizeof(storage) % 16 == 0 and a fitting tile
    step_fn pair;            // variant 2: flat cell pairs (two cells of the flat index per thread), any nx
    // fixed-point storage: the same kernels with a per-velocity reference shift in the codec
    // (its extra constants cost instructions, so the plain set keeps uniform ones); else null
    const struct KernelSet *shifted;
};

// Defined in the instantiation units, one per lattice.
const KernelSet *kernels_d2q9(int K, lbm_storage st);
const KernelSet *kernels_d3q15(int K, lbm_storage st);
const KernelSet *kernels_d3q19(int K, lbm_storage st);
const KernelSet *kernels_d3q27(int K, lbm_storage st);
const KernelSet *kernels_d3q39(int K, lbm_storage st);

// Shared helpers of the C-ABI units (defined in lbm_api.cu).
lbm_status set_error(lbm_status s, const char *msg);
lbm_status set_cuda_error(cudaError_t e, const char *what);
bool lattice_query(lbm_lattice lat, int *D, int *Q, int *maxc, int *kmax);
size_t storage_bytes(lbm_storage st);
const KernelSet *kernel_set(lbm_lattice lat, int K, lbm_storage st);

constexpr int kReduceBlocks = 1216;  // 8 x 152 SMs
constexpr int kReduceThreads = 256;

std::string dims_check(lbm_lattice lat, const int64_t *dims);  // empty when valid

}  // namespace lbm
