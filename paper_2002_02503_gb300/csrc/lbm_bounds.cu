// lbm_bounds.cu -- host side of the bounds-check build: which build this library is, and a
// host walk of the register-pull step's index arithmetic that needs no GPU.
//
// The walk restates, for every thread of one launch of the register-pull step (V cells per
// thread, the grid the launcher uses), the offsets its loads and stores compute inside a
// velocity plane, and checks each span with span_in -- the test the bounds-check build's
// kernels apply before every access.  It follows the x-shift scheme of the plain storage
// forms: whole-chunk loads on D3Q39 (the reference-velocity forms use them on every lattice,
// with the same offsets in their reference planes), shuffles with direct loads at the warp and
// row edges on the other lattices.  With a consistent plane size (P = nx*ny*nz) nothing
// falls outside; with an inconsistent dims/P pair the walk counts the accesses the device
// guard would skip and record.
#include <cuda_runtime.h>

#include "lbm_internal.h"

using namespace lbm;

namespace {

int wrap_host(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
int floordiv_host(int e, int V) { return e >= 0 ? e / V : -((-e + V - 1) / V); }

}  // namespace

extern "C" int lbm_bounds_checked(void) { return kBoundsCheck ? 1 : 0; }

extern "C" int64_t lbm_bounds_walk(lbm_lattice lattice, int V, const int64_t dims[3], int64_t P, int64_t *accesses) {
    if (accesses) *accesses = 0;
    int D = 0, Q = 0, maxc = 0, kmax = 0;
    if (!dims || !lattice_query(lattice, &D, &Q, &maxc, &kmax)) return -1;
    if (v_index(V) < 0 || !dims_check(lattice, dims).empty() || dims[0] % V) return -1;
    int c[3 * kQMax];
    if (lbm_lattice_info(lattice, nullptr, nullptr, c, nullptr, nullptr, nullptr) != LBM_OK) return -1;
    const int nx = int(dims[0]), ny = int(dims[1]), nz = int(dims[2]);
    const int ncx = nx / V;
    const long long total = (long long)ncx * ny;  // threads per z-plane (grid.x * block covers it)
    const int kMaxDl = (maxc + V - 1) / V;
    // the x-shift scheme of the plain storage forms: whole-chunk loads on the max|c| >= 2 set,
    // shuffles with direct loads at warp and row edges on the others
    const bool chunk_loads = V > 1 && maxc >= 2;
    long long bad = 0, n = 0;
    auto check = [&](long long first, int len) {
        ++n;
        if (!span_in(first, len, P)) ++bad;
    };
    for (int z = 0; z < nz; ++z)
        for (long long tt = 0; tt < (total + 31) / 32 * 32; ++tt) {  // whole warps, as launched
            const bool active = tt < total;
            const long long t = active ? tt : total - 1;  // inactive lanes compute on the last thread
            const int lane = int(tt & 31);
            const int y = int(t / ncx);
            const int chunk = int(t - (long long)y * ncx);
            const int x0 = chunk * V;
            for (int i = 0; i < Q; ++i) {
                const int cx = c[3 * i], cy = c[3 * i + 1], cz = c[3 * i + 2];
                const long long roff = (long long)(wrap_host(z - cz, nz) * ny + wrap_host(y - cy, ny)) * nx;
                if (V == 1) {
                    check(roff + wrap_host(x0 - cx, nx), 1);
                    continue;
                }
                if (chunk_loads) {
                    // every chunk that holds a shifted value, loaded whole (wrapped by whole chunks)
                    for (int dl = -kMaxDl; dl <= kMaxDl; ++dl) {
                        bool need = false;
                        for (int j = 0; j < V; ++j) need = need || floordiv_host(j - cx, V) == dl;
                        if (need) check(roff + (long long)wrap_host(chunk + dl, ncx) * V, V);
                    }
                    continue;
                }
                check(roff + x0, V);  // the row vector
                for (int j = 0; j < V; ++j) {
                    const int e = j - cx;
                    const int dl = floordiv_host(e, V);
                    if (dl == 0 || cx == 0) continue;
                    const bool ok = lane + dl >= 0 && lane + dl <= 31 && chunk + dl >= 0 && chunk + dl < ncx &&
                                    dl >= -kMaxDl && dl <= kMaxDl;
                    if (!ok) check(roff + wrap_host(x0 + e, nx), 1);  // the direct load at a warp or row edge
                }
            }
            if (active) check((long long)(z * ny + y) * nx + x0, V);  // the stores
        }
    if (accesses) *accesses = n;
    return bad;
}
