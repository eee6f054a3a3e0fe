// Plan construction and the C ABI (include/p3dfft_gb300.h).
//
// A plan fixes, for each direction, the sequence of stage launches of the
// P3DFFT method (Sect. 2, Fig. 2): X real-to-complex, Y complex, Z complex /
// Chebyshev / empty, each a batched 1D transform over every line of the
// volume, and the buffers each stage reads and writes.  The paper's
// pencil re-orientations (Sect. 3.3) become the stage kernels' load and store
// addressing; the STRIDE1 Z-pencil layout (ZYX, Table 1) is produced by the
// Z stage's store and consumed by the inverse Z stage's load.
//
// The host builds every table in FP64 (roots of unity by exact integer
// reduction of the angle to an octant, Bluestein chirps with j^2 reduced mod
// 2n in integers) and rounds it once to the plan's precision.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/p3dfft_gb300.h"
#include "p3_internal.h"

using p3::LineMap;
using p3::StageArgs;

namespace {

enum Buf { BUF_IN = 0, BUF_OUT = 1, BUF_WS = 2 };

struct Stage {
    StageArgs a;
    int src, dst;       // Buf roles
    const char* name;
    double bytes;       // algorithmic HBM bytes of one launch
    bool fused;         // plane-fused X + Y launch (f); a is its X stage
    p3::PlaneArgs f;
};

struct TableKey {
    int kind;  // 0 roots, 1 chirp, 2 bhat
    long long n, m;
    bool operator<(const TableKey& o) const
    {
        if (kind != o.kind) return kind < o.kind;
        if (n != o.n) return n < o.n;
        return m < o.m;
    }
};

}  // namespace

struct p3_plan_s {
    int nx, ny, nz, H;
    p3_precision prec;
    p3_ttype tt[3];
    p3_layout layout;
    int device;
    size_t csize;  // bytes per complex element
    void* dtab;
    // st[0] forward, st[1] inverse, st[2] the inverse used while a Z hook is
    // set (EMPTY third dimension: a Z copy into the work buffer comes first)
    std::vector<Stage> st[3];
    // the stage lists before plane fusion, with their tables (the generic
    // stages of the batched persistent launch start from these)
    std::vector<Stage> st_unfused[2];
    p3_z_hook hook;
    void* hook_user;
    size_t ctr_off;     // byte offset of the fused kernels' counters in the workspace
    unsigned* derr;     // device word: a bounded wait of a fused kernel gave up
    unsigned spin_limit, wait_extra;
    int fused_lag_default[3];
    size_t ws_bytes;
    double scale;
    bool padded;  // real rows of 2H values (in-place capable, XYZ layout)
    void* events[8];
    bool timing;
    std::string desc;
};

namespace {

const long double kPi = 3.141592653589793238462643383279502884L;

// exp(-2 pi i k / n) in FP64: the angle is reduced exactly to octant o and an
// offset x in [0, pi/4] before cosl/sinl, then rotated back by symmetry.
std::complex<double> unit_root(long long k, long long n)
{
    k %= n;
    if (k < 0) k += n;
    const long long o = (8 * k) / n;
    const long long r = 8 * k - o * n;  // angle = (pi/4) (o + r/n)
    long double c, s;                   // cos / sin of the angle
    if ((o & 1) == 0) {
        const long double x = (kPi / 4) * (long double)r / (long double)n;
        const long double cx = cosl(x), sx = sinl(x);
        switch (o / 2) {
        case 0: c = cx; s = sx; break;
        case 1: c = -sx; s = cx; break;
        case 2: c = -cx; s = -sx; break;
        default: c = sx; s = -cx; break;
        }
    } else {
        const long double y = (kPi / 4) * (long double)(n - r) / (long double)n;  // (o+1) pi/4 - angle
        const long double cy = cosl(y), sy = sinl(y);
        switch ((o + 1) / 2) {
        case 1: c = sy; s = cy; break;
        case 2: c = -cy; s = sy; break;
        case 3: c = -sy; s = -cy; break;
        default: c = cy; s = -sy; break;
        }
    }
    return std::complex<double>((double)c, -(double)s);
}

// In-place iterative radix-2 DFT (exp(-2 pi i ...)) in long double, for the
// Bluestein filter spectrum at plan time; m is a power of two.
void host_dft_pow2(std::vector<std::complex<long double>>& a)
{
    const size_t m = a.size();
    for (size_t i = 1, j = 0; i < m; ++i) {
        size_t bit = m >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= m; len <<= 1) {
        for (size_t i = 0; i < m; i += len) {
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w = unit_root((long long)k, (long long)len);
                const std::complex<long double> wl((long double)w.real(), (long double)w.imag());
                const std::complex<long double> u = a[i + k], v = a[i + k + len / 2] * wl;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

// FP32 generic stages factor their lengths into composite radices (1) or
// the native ones only (0).
#ifndef P3_GEN_COMPOSITE
#define P3_GEN_COMPOSITE 1
#endif
// Radix sequence for n (16s first, then 8/4/2, then 3, 5, 7).  With
// composite = true (FP32 plans) and a factor 3, 5 or 7 in n, the sequence
// instead takes the fewest passes from the native radices and the composite
// register butterflies 6 .. 28, ties going to the one whose smallest radix is
// largest, largest radix first.  Returns false when n has a prime factor
// above 7.
bool factor(int n, std::vector<int>& rad, bool composite = false)
{
    rad.clear();
    int m = n;
    int e2 = 0, e3 = 0, e5 = 0, e7 = 0;
    while (m > 1 && m % 2 == 0) { m /= 2; ++e2; }
    while (m > 1 && m % 3 == 0) { m /= 3; ++e3; }
    while (m > 1 && m % 5 == 0) { m /= 5; ++e5; }
    while (m > 1 && m % 7 == 0) { m /= 7; ++e7; }
    if (m != 1) return false;
    if (composite && e3 + e5 + e7 > 0) {
        // radices as exponent vectors (2, 3, 5, 7)
        static const int kRad[][5] = {
            {28, 2, 0, 0, 1}, {27, 0, 3, 0, 0}, {25, 0, 0, 2, 0}, {24, 3, 1, 0, 0}, {21, 0, 1, 0, 1},
            {20, 2, 0, 1, 0}, {18, 1, 2, 0, 0}, {16, 4, 0, 0, 0}, {15, 0, 1, 1, 0}, {14, 1, 0, 0, 1},
            {12, 2, 1, 0, 0}, {10, 1, 0, 1, 0}, {9, 0, 2, 0, 0},  {8, 3, 0, 0, 0},  {7, 0, 0, 0, 1},
            {6, 1, 1, 0, 0},  {5, 0, 0, 1, 0},  {4, 2, 0, 0, 0},  {3, 0, 1, 0, 0},  {2, 1, 0, 0, 0}};
        struct Best {
            int passes, minr;
            std::vector<int> seq;
        };
        std::map<long long, Best> memo;
        std::function<Best(int, int, int, int)> best = [&](int a, int b, int c, int d) -> Best {
            if (a + b + c + d == 0) return Best{0, 1 << 30, {}};
            const long long key = (((long long)a * 64 + b) * 64 + c) * 64 + d;
            auto it = memo.find(key);
            if (it != memo.end()) return it->second;
            Best r{1 << 30, 0, {}};
            for (const auto& k : kRad) {
                if (k[1] > a || k[2] > b || k[3] > c || k[4] > d) continue;
                if (k[0] > p3::kMaxCompositeRadix && k[0] != 16) continue;
                Best t = best(a - k[1], b - k[2], c - k[3], d - k[4]);
                const int passes = t.passes + 1, minr = std::min(t.minr, k[0]);
                if (passes < r.passes || (passes == r.passes && minr > r.minr)) {
                    t.seq.push_back(k[0]);
                    r = Best{passes, minr, t.seq};
                }
            }
            memo[key] = r;
            return r;
        };
        rad = best(e2, e3, e5, e7).seq;
        std::sort(rad.begin(), rad.end(), std::greater<int>());
        return (int)rad.size() <= p3::kMaxPasses;
    }
    m = n;
    while (m % 16 == 0) { rad.push_back(16); m /= 16; }
    if (m % 8 == 0) { rad.push_back(8); m /= 8; }
    if (m % 4 == 0) { rad.push_back(4); m /= 4; }
    if (m % 2 == 0) { rad.push_back(2); m /= 2; }
    for (int p : {3, 5, 7})
        while (m % p == 0) { rad.push_back(p); m /= p; }
    return m == 1 && (int)rad.size() <= p3::kMaxPasses;
}

// Every radix has a butterfly in the generic kernel of the plan's precision
// (a pass of any other radix would be skipped there).
bool radices_supported(const std::vector<int>& rad, bool composite)
{
    for (int r : rad) {
        const bool native = r == 2 || r == 3 || r == 4 || r == 5 || r == 7 || r == 8 || r == 16;
        const bool comp = composite && r <= p3::kMaxCompositeRadix &&
                          (r == 6 || r == 9 || r == 10 || r == 12 || r == 14 || r == 15 || r == 18 || r == 20 ||
                           r == 21 || r == 24 || r == 25 || r == 27 || r == 28);
        if (!native && !comp) return false;
    }
    return true;
}

// Threads per line of the generic kernel: each thread takes about kVmax
// values per pass (the passes loop over butterflies, so any count works);
// with P3_GEN_TPL_MAXR, at least the largest radix's worth, so that the
// passes of a composite radix above kVmax keep every thread busy.
#ifndef P3_GEN_TPL_MAXR
#define P3_GEN_TPL_MAXR 0
#endif
int threads_per_line(int n, const std::vector<int>& rad)
{
    int vmax = p3::kVmax;
    if (P3_GEN_TPL_MAXR)
        for (int r : rad) vmax = std::max(vmax, r);
    int tpl = (n + vmax - 1) / vmax;
    if (tpl < 1) tpl = 1;
    if (tpl > p3::kMaxThreads) tpl = p3::kMaxThreads;
    return tpl;
}

int pow2_floor(long long v)
{
    int p = 1;
    while ((long long)p * 2 <= v) p *= 2;
    return p;
}

long long pow2_ceil(long long v)
{
    long long p = 1;
    while (p < v) p *= 2;
    return p;
}

struct TableSet {
    std::map<TableKey, size_t> offs;  // byte offsets into the device block
    std::vector<std::complex<double>> vals;
    size_t add(const TableKey& k, std::vector<std::complex<double>>&& v)
    {
        auto it = offs.find(k);
        if (it != offs.end()) return it->second;
        const size_t off = vals.size();
        vals.insert(vals.end(), v.begin(), v.end());
        offs[k] = off;
        return off;
    }
};

size_t roots_table(TableSet& T, long long n)
{
    std::vector<std::complex<double>> v((size_t)n);
    for (long long k = 0; k < n; ++k) v[(size_t)k] = unit_root(k, n);
    return T.add(TableKey{0, n, 0}, std::move(v));
}

// Per-pass twiddles of a power-of-two line of n points with E values per
// thread, laid out for row-style lanes (see rtw_off in p3_pow2.cuh): pass
// p >= 1 (NS = the product of the earlier radices, radix R, step n/(NS R))
// stores, at (r - 1) NS + q, the entry the roots table of length tn gives at
// index q step r (tn / n).
size_t row_tw_table(TableSet& T, long long n, int E, long long tn)
{
    int logn = 0, loge = 0;
    while ((1LL << logn) < n) ++logn;
    while ((1 << loge) < E) ++loge;
    const int nfull = logn / loge;
    const long long rem = 1LL << (logn - nfull * loge);
    const int npass = nfull + (rem > 1 ? 1 : 0);
    std::vector<std::complex<double>> v;
    long long ns = 1;
    for (int p = 0; p < npass; ++p) {
        const long long R = p < nfull ? E : rem;
        if (p >= 1) {
            const long long step = n / (ns * R);
            for (long long r = 1; r < R; ++r)
                for (long long q = 0; q < ns; ++q) v.push_back(unit_root(q * step * r * (tn / n), tn));
        }
        ns *= R;
    }
    return T.add(TableKey{3, n * 64 + E, tn}, std::move(v));
}

size_t chirp_table(TableSet& T, long long n)
{
    std::vector<std::complex<double>> v((size_t)n);
    for (long long j = 0; j < n; ++j) v[(size_t)j] = unit_root((j * j) % (2 * n), 2 * n);
    return T.add(TableKey{1, n, 0}, std::move(v));
}

size_t bhat_table(TableSet& T, long long n, long long m)
{
    std::vector<std::complex<long double>> b((size_t)m, std::complex<long double>(0, 0));
    for (long long j = 0; j < n; ++j) {
        const std::complex<double> c = std::conj(unit_root((j * j) % (2 * n), 2 * n));
        const std::complex<long double> cl((long double)c.real(), (long double)c.imag());
        b[(size_t)j] = cl;
        if (j) b[(size_t)(m - j)] = cl;
    }
    host_dft_pow2(b);
    std::vector<std::complex<double>> v((size_t)m);
    for (long long k = 0; k < m; ++k)
        v[(size_t)k] = std::complex<double>((double)(b[(size_t)k].real() / m), (double)(b[(size_t)k].imag() / m));
    return T.add(TableKey{2, n, m}, std::move(v));
}

// Pointer-valued table fields hold byte offsets (+1, 0 = none) until the
// device block exists.
struct Pending {
    size_t tw = 0, tw2 = 0, chirp = 0, bhat = 0, twm = 0, twr = 0;
};

// Line-FFT set-up: native radices over nfft, else Bluestein over m.
// Returns P3_ERR_UNSUPPORTED for lines beyond the shared-memory limit.
p3_status line_setup(StageArgs& a, Pending& pend, TableSet& T, int twn_native, bool composite)
{
    std::vector<int> rad;
    a.blue = 0;
    a.npass = 0;
    a.mpass = 0;
    a.m = 0;
    if (a.nfft <= 1) {
        a.tpl = 1;
        return P3_OK;
    }
    if (factor(a.nfft, rad, composite)) {
        if (a.nfft > p3::kMaxLine) return P3_ERR_UNSUPPORTED;
        if (!radices_supported(rad, composite)) return P3_ERR_UNSUPPORTED;
        a.npass = (int)rad.size();
        for (int i = 0; i < a.npass; ++i) a.rad[i] = rad[i];
        a.tpl = threads_per_line(a.nfft, rad);
        if (a.tpl > p3::kMaxThreads) return P3_ERR_UNSUPPORTED;
        a.twn = twn_native;
        pend.tw = roots_table(T, twn_native) + 1;
        return P3_OK;
    }
    const long long m = pow2_ceil(2LL * a.nfft - 1);
    if (m > p3::kMaxLine) return P3_ERR_UNSUPPORTED;
    factor((int)m, rad);
    a.blue = 1;
    a.m = (int)m;
    a.mpass = (int)rad.size();
    for (int i = 0; i < a.mpass; ++i) a.mrad[i] = rad[i];
    a.tpl = threads_per_line((int)m, rad);
    if (a.tpl > p3::kMaxThreads) return P3_ERR_UNSUPPORTED;
    pend.chirp = chirp_table(T, a.nfft) + 1;
    pend.bhat = bhat_table(T, a.nfft, m) + 1;
    pend.twm = roots_table(T, m) + 1;
    return P3_OK;
}

// Lines per CTA, pitch, threads and shared memory of a stage.
// Tile shape of the generic kernel: B lines per CTA (a power of two) so that
// the ping-pong buffers fit 100 KB, LDB the shared-memory pitch.
// Shared memory a generic-kernel tile may take (bytes).
#ifndef P3_GEN_SMEM_CAP
#define P3_GEN_SMEM_CAP (100 * 1024)
#endif
void generic_tile_setup(StageArgs& a, size_t csize, size_t cap = P3_GEN_SMEM_CAP, int maxt = p3::kGenThreads)
{
    const int len = a.blue ? a.m : (a.nfft > 0 ? a.nfft : 1);
    const bool elem = a.in_elem_fast || a.out_elem_fast;
    int B = pow2_floor(maxt / a.tpl);
    if (B < 1) B = 1;
    while (B > 1 && 2 * (size_t)len * (size_t)(B + 1) * csize > cap) B /= 2;
    const long long lim = pow2_ceil(a.nlines > 0 ? a.nlines : 1);
    if (B > lim) B = (int)lim;
    a.B = B;
    a.LDB = (elem && (B % 2 == 0)) ? B + 1 : B;
    int th = B * a.tpl;
    th = (th + 31) / 32 * 32;
    a.threads = th;
    a.smem = 2 * (size_t)len * (size_t)a.LDB * csize;  // ping-pong buffers
    a.kern = p3::KIND_GENERIC;
    a.tc = 0;
    a.tma = 0;
}

void tile_setup(StageArgs& a, size_t csize, unsigned flags)
{
    generic_tile_setup(a, csize);
    p3::pow2_configure(a, csize, !(flags & P3_FLAG_NO_TMA));
    if (flags & P3_FLAG_TC_SPLIT) p3::tc_configure(a, csize);
}

LineMap rows(long long nlines, long long pitch) { return LineMap{nlines > 0 ? nlines : 1, 0, pitch, 1}; }

const char* op_name(int op)
{
    switch (op) {
    case p3::OP_C2C: return "c2c";
    case p3::OP_R2C_HALF: return "r2c_half";
    case p3::OP_R2C_PAIR: return "r2c_pair";
    case p3::OP_C2R_HALF: return "c2r_half";
    case p3::OP_C2R_PAIR: return "c2r_pair";
    case p3::OP_DCT1: return "dct1";
    case p3::OP_DST1: return "dst1";
    default: return "copy";
    }
}

const char* kern_name(int k, int tc, int tma = 0)
{
    if (tc) return "tc_split_col";
    if (tma == 2) return "pow2_zrow_bulk";
    if (tma) return "pow2_col_zyx_store_tma";
    switch (k) {
    case p3::KIND_COL_DD: return "pow2_col";
    case p3::KIND_COL_DS: return "pow2_col_zyx_store";
    case p3::KIND_COL_SD: return "pow2_col_zyx_load";
    case p3::KIND_ROW_R2C: return "pow2_row_r2c";
    case p3::KIND_ROW_C2R: return "pow2_row_c2r";
    default: return "generic";
    }
}

// Whether a line of n points has a kernel: n <= 1, or a 2/3/5/7-smooth n up
// to the longest native line, or a Bluestein length whose padded transform
// fits.  n is 64-bit so that the extended lengths 2(Nz - 1) and 2(Nz + 1)
// of the Chebyshev and sine transforms cannot wrap for any int Nz.
bool smooth_or_small(long long n)
{
    std::vector<int> r;
    if (n <= 1) return true;
    if (n > p3::kMaxLine) return false;  // longer than any native or Bluestein-padded line
    if (factor((int)n, r)) return true;
    return pow2_ceil(2LL * n - 1) <= p3::kMaxLine;
}


bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace

extern "C" {
static p3_status run(p3_plan P, int dir, const void* in, void* out, void* ws, void* stream);
}

// P3_FLAG_TUNE: for each direction with a plane-fused launch, time the
// candidates -- the fused launch at a few queue lags and the separate X and
// Y launches (with plain planes) -- on temporary buffers of the transform's
// size, and keep the fastest.  The candidates compute the same result.
static p3_status tune(p3_plan P, std::vector<Stage> (&unfused)[3], std::string& report)
{
    const size_t rowr = P->padded ? 2 * (size_t)P->H : (size_t)P->nx;
    const size_t nreal = rowr * P->ny * P->nz * (P->csize / 2);
    const size_t ncplx = (size_t)P->H * P->ny * P->nz * P->csize;
    const size_t nbuf = nreal > ncplx ? nreal : ncplx;
    void *a = NULL, *b = NULL, *w = NULL;
    cudaStream_t st = NULL;
    cudaEvent_t e0 = NULL, e1 = NULL;
    p3_status rc = P3_OK;
    if (cudaMalloc(&a, nbuf) != cudaSuccess || cudaMalloc(&b, nbuf) != cudaSuccess ||
        cudaMalloc(&w, P->ws_bytes) != cudaSuccess)
        rc = P3_ERR_NOMEM;
    if (rc == P3_OK && (cudaMemset(a, 0x3c, nbuf) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = P3_ERR_CUDA;
    const bool timing = P->timing;
    P->timing = false;
    for (int d = 0; d < 2 && rc == P3_OK; ++d) {
        int fi = -1;
        for (size_t i = 0; i < P->st[d].size(); ++i)
            if (P->st[d][i].fused) fi = (int)i;
        if (fi < 0) continue;
        const std::vector<Stage> fused = P->st[d];
        const int lag0 = fused[(size_t)fi].f.lag, np = fused[(size_t)fi].f.nplanes;
        std::vector<int> lags;  // 0: separate X and Y launches
        for (int L : {lag0, lag0 / 2, (3 * lag0) / 2, 2 * lag0}) {
            const int l = L < 1 ? 1 : (L > np ? np : L);
            if (std::find(lags.begin(), lags.end(), l) == lags.end()) lags.push_back(l);
        }
        lags.push_back(0);
        float best = 1e30f;
        int pick = lag0;
        std::string line = std::string(d == 0 ? "fwd" : "bwd") + " tuned:";
        for (int L : lags) {
            if (L == 0) {
                P->st[d] = unfused[d];
            } else {
                P->st[d] = fused;
                P->st[d][(size_t)fi].f.lag = L;
            }
            const void* in = d == 0 ? a : b;
            void* out = d == 0 ? b : a;
            float ms = 0.f;
            for (int rep = 0; rep < 4 && rc == P3_OK; ++rep) {
                if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = P3_ERR_CUDA;
                if (rc == P3_OK) rc = run(P, d, in, out, w, st);
            }
            if (rc == P3_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = P3_ERR_CUDA;
            if (rc != P3_OK) break;
            ms /= 3.f;
            char buf[64];
            snprintf(buf, sizeof(buf), " %s=%.3fms", L ? ("lag" + std::to_string(L)).c_str() : "separate", ms);
            line += buf;
            if (ms < best) {
                best = ms;
                pick = L;
            }
        }
        if (rc != P3_OK) break;
        if (pick == 0) {
            P->st[d] = unfused[d];
        } else {
            P->st[d] = fused;
            P->st[d][(size_t)fi].f.lag = pick;
            P->fused_lag_default[d] = pick;
        }
        report += line + " -> " + (pick ? "lag" + std::to_string(pick) : std::string("separate")) + "\n";
    }
    P->timing = timing;
    if (rc == P3_OK && p3_plan_wait_status(P) != P3_OK) rc = P3_ERR_TIMEOUT;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (w) cudaFree(w);
    cudaGetLastError();
    return rc;
}

// P3_FLAG_TUNE for the generic stages (lengths that are not powers of two,
// Bluestein lines excepted): time each stage alone under a few radix orders
// of its factorisation and tile heights B, B / 2, B / 4 on temporary
// buffers, and keep the fastest.  Any order is the same DFT with the same
// root table; only rounding differs.
static p3_status tune_generic(p3_plan P, std::string& report)
{
    const size_t rowr = P->padded ? 2 * (size_t)P->H : (size_t)P->nx;
    const size_t nreal = rowr * P->ny * P->nz * (P->csize / 2);
    const size_t ncplx = (size_t)P->H * P->ny * P->nz * P->csize;
    const size_t nbuf = std::max(std::max(nreal, ncplx), P->ws_bytes) + 256;
    bool any = false;
    for (int d = 0; d < 2; ++d)
        for (const Stage& st : P->st[d])
            if (!st.fused && st.a.kern == p3::KIND_GENERIC && !st.a.blue && st.a.op != p3::OP_COPY && st.a.npass > 1)
                any = true;
    if (!any) return P3_OK;
    void* buf[3] = {NULL, NULL, NULL};
    cudaStream_t sm = NULL;
    cudaEvent_t e0 = NULL, e1 = NULL;
    p3_status rc = P3_OK;
    for (int i = 0; i < 3 && rc == P3_OK; ++i)
        if (cudaMalloc(&buf[i], nbuf) != cudaSuccess) rc = P3_ERR_NOMEM;
    for (int i = 0; i < 3 && rc == P3_OK; ++i)
        if (cudaMemset(buf[i], 0x3c, nbuf) != cudaSuccess) rc = P3_ERR_CUDA;
    if (rc == P3_OK && (cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = P3_ERR_CUDA;
    for (int d = 0; d < 2 && rc == P3_OK; ++d) {
        for (size_t si = 0; si < P->st[d].size() && rc == P3_OK; ++si) {
            Stage& st = P->st[d][si];
            StageArgs& a0 = st.a;
            if (st.fused || a0.kern != p3::KIND_GENERIC || a0.blue || a0.op == p3::OP_COPY || a0.npass <= 1) continue;
            // candidate radix orders: as factored, reversed, ascending, and
            // each rotation of the factored order
            std::vector<std::vector<int>> orders;
            std::vector<int> base(a0.rad, a0.rad + a0.npass);
            auto add_order = [&](const std::vector<int>& o) {
                if (std::find(orders.begin(), orders.end(), o) == orders.end()) orders.push_back(o);
            };
            add_order(base);
            add_order(std::vector<int>(base.rbegin(), base.rend()));
            std::vector<int> asc = base;
            std::sort(asc.begin(), asc.end());
            add_order(asc);
            for (size_t k = 1; k < base.size(); ++k) {
                std::vector<int> rot(base.begin() + k, base.end());
                rot.insert(rot.end(), base.begin(), base.begin() + k);
                add_order(rot);
            }
            float best = 1e30f;
            StageArgs pick = a0;
            std::string line = std::string(d == 0 ? "fwd " : "bwd ") + st.name + " tuned:";
            for (const auto& o : orders) {
                for (int shrink = 0; shrink < 3 && rc == P3_OK; ++shrink) {
                    StageArgs a = a0;
                    for (size_t k = 0; k < o.size(); ++k) a.rad[k] = o[k];
                    generic_tile_setup(a, P->csize);
                    if ((a.B >> shrink) < 1) break;
                    if (shrink) {
                        a.B >>= shrink;
                        const bool elem = a.in_elem_fast || a.out_elem_fast;
                        a.LDB = (elem && (a.B % 2 == 0)) ? a.B + 1 : a.B;
                        a.threads = (a.B * a.tpl + 31) / 32 * 32;
                        const int len = a.nfft > 0 ? a.nfft : 1;
                        a.smem = 2 * (size_t)len * (size_t)a.LDB * P->csize;
                    }
                    a.src = buf[st.src];
                    a.dst = buf[st.dst];
                    a.err = P->derr;
                    float ms = 0.f;
                    for (int rep = 0; rep < 4 && rc == P3_OK; ++rep) {
                        if (rep == 1 && cudaEventRecord(e0, sm) != cudaSuccess) rc = P3_ERR_CUDA;
                        const cudaError_t e = P->prec == P3_F32 ? p3::launch_stage_f32(a, sm) : p3::launch_stage_f64(a, sm);
                        if (e != cudaSuccess) rc = P3_ERR_CUDA;
                    }
                    if (rc == P3_OK && (cudaEventRecord(e1, sm) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                        rc = P3_ERR_CUDA;
                    if (rc != P3_OK) break;
                    ms /= 3.f;
                    std::string rs;
                    for (size_t k = 0; k < o.size(); ++k) rs += (k ? "x" : "") + std::to_string(o[k]);
                    char b[96];
                    snprintf(b, sizeof(b), " %s/B%d=%.4fms", rs.c_str(), a.B, ms);
                    line += b;
                    if (ms < best) {
                        best = ms;
                        pick = a;
                    }
                }
            }
            if (rc != P3_OK) break;
            pick.src = NULL;
            pick.dst = NULL;
            a0 = pick;
            std::string rs;
            for (int k = 0; k < a0.npass; ++k) rs += (k ? "x" : "") + std::to_string(a0.rad[k]);
            report += line + " -> " + rs + "/B" + std::to_string(a0.B) + "\n";
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sm) cudaStreamDestroy(sm);
    for (void* b : buf)
        if (b) cudaFree(b);
    cudaGetLastError();
    return rc;
}

extern "C" {

const char* p3_status_string(p3_status s)
{
    switch (s) {
    case P3_OK: return "ok";
    case P3_ERR_INVALID: return "invalid argument";
    case P3_ERR_UNSUPPORTED: return "unsupported";
    case P3_ERR_NOMEM: return "out of memory";
    case P3_ERR_CUDA: return "CUDA error";
    case P3_ERR_TIMEOUT: return "device wait timed out";
    case P3_ERR_WORKSPACE: return "workspace required";
    case P3_ERR_HOOK: return "user Z hook failed";
    default: return "unknown status";
    }
}

int p3_version(void) { return P3_VERSION; }

p3_status p3_plan_create(p3_plan* out, int nx, int ny, int nz, p3_precision prec, const p3_ttype ttype[3],
                         p3_layout out_layout, unsigned flags)
{
    if (!out) return P3_ERR_INVALID;
    *out = NULL;
    if (!ttype || nx < 1 || ny < 1 || nz < 1 ||
        (flags & ~(unsigned)(P3_FLAG_TC_SPLIT | P3_FLAG_PADDED_REAL | P3_FLAG_NO_FUSE | P3_FLAG_TUNE |
                             P3_FLAG_NO_TMA)))
        return P3_ERR_INVALID;
    if (prec != P3_F32 && prec != P3_F64) return P3_ERR_INVALID;
    if (out_layout != P3_LAYOUT_ZYX && out_layout != P3_LAYOUT_XYZ) return P3_ERR_INVALID;
    for (int d = 0; d < 3; ++d)
        if (ttype[d] != P3_FFT && ttype[d] != P3_CHEB && ttype[d] != P3_EMPTY && ttype[d] != P3_SINE)
            return P3_ERR_INVALID;
    if (ttype[0] != P3_FFT) return P3_ERR_UNSUPPORTED;
    if (ttype[1] == P3_CHEB || ttype[1] == P3_SINE) return P3_ERR_UNSUPPORTED;
    if (ttype[2] == P3_CHEB && nz < 2) return P3_ERR_INVALID;
    const bool padded = (flags & P3_FLAG_PADDED_REAL) != 0;
    if (padded && out_layout != P3_LAYOUT_XYZ) return P3_ERR_UNSUPPORTED;
    // per-line length limits
    if (!smooth_or_small(nx % 2 == 0 ? nx / 2 : nx)) return P3_ERR_UNSUPPORTED;
    if (ttype[1] == P3_FFT && !smooth_or_small(ny)) return P3_ERR_UNSUPPORTED;
    if (ttype[2] == P3_FFT && !smooth_or_small(nz)) return P3_ERR_UNSUPPORTED;
    if (ttype[2] == P3_CHEB && !smooth_or_small(2LL * (nz - 1))) return P3_ERR_UNSUPPORTED;
    if (ttype[2] == P3_SINE && !smooth_or_small(2LL * ((long long)nz + 1))) return P3_ERR_UNSUPPORTED;

    p3_plan P = new (std::nothrow) p3_plan_s();
    if (!P) return P3_ERR_NOMEM;
    P->nx = nx; P->ny = ny; P->nz = nz; P->H = nx / 2 + 1;
    P->prec = prec;
    for (int d = 0; d < 3; ++d) P->tt[d] = ttype[d];
    P->layout = out_layout;
    P->padded = padded;
    P->csize = prec == P3_F32 ? 8 : 16;
    P->dtab = NULL;
    P->hook = NULL;
    P->hook_user = NULL;
    P->ctr_off = 0;
    P->derr = NULL;
    P->spin_limit = 1u << 23;
    P->wait_extra = 0;
    P->timing = false;
    memset(P->events, 0, sizeof(P->events));
    const long long H = P->H, NY = ny, NZ = nz, NX = nx;
    const size_t e = P->csize / 2;
    const long long RP = padded ? 2 * H : NX;             // real row pitch (elements)
    const double creal = (double)e * NX * NY * NZ;        // bytes of the real array
    const double ccplx = (double)P->csize * H * NY * NZ;  // bytes of the complex array

    P->scale = (double)nx;
    P->scale *= ttype[1] == P3_FFT ? (double)ny : 1.0;
    P->scale *= ttype[2] == P3_FFT    ? (double)nz
                : ttype[2] == P3_CHEB ? 2.0 * (nz - 1)
                : ttype[2] == P3_SINE ? 2.0 * (nz + 1)
                                      : 1.0;

    TableSet T;
    std::vector<Pending> pend[3];
    p3_status rc = P3_OK;

    const LineMap mapY = LineMap{H, NY * H, 1, H};
    const LineMap mapZxyz = LineMap{H * NY, 0, 1, NY * H};
    const LineMap mapZzyx = LineMap{H, NZ, NY * NZ, 1};
    const bool zyx = out_layout == P3_LAYOUT_ZYX;

    auto base_args = [&](int op, int n_in, int n_out, int nfft, int sign, long long nlines, LineMap in,
                         LineMap outm) {
        StageArgs a;
        memset(&a, 0, sizeof(a));
        a.op = op; a.n_in = n_in; a.n_out = n_out; a.nfft = nfft; a.sign = sign;
        a.nlines = nlines; a.in = in; a.out = outm;
        a.in_elem_fast = in.es == 1;
        a.out_elem_fast = outm.es == 1;
        return a;
    };
    // odd Nx: the X stage takes its real rows in pairs, one complex FFT of
    // length Nx per two rows (line L: rows 2L and 2L + 1)
    auto pair_args = [&](int op, int n_in, int n_out, int sign, LineMap in, LineMap outm) {
        StageArgs a = base_args(op, n_in, n_out, nx, sign, (NY * NZ + 1) / 2, in, outm);
        a.nrows = NY * NZ;
        return a;
    };
    auto push = [&](int dir, StageArgs a, int src, int dst, const char* name, double bytes, int twn) {
        Pending pd;
        if (rc != P3_OK) return;
        if (a.op == p3::OP_R2C_HALF || a.op == p3::OP_C2R_HALF) {
            pd.tw2 = roots_table(T, NX) + 1;
        }
        if (a.op != p3::OP_COPY) {
            rc = line_setup(a, pd, T, twn, prec == P3_F32 && P3_GEN_COMPOSITE);
            if (rc != P3_OK) return;
            // row-style twiddles for power-of-two lines (E as the row kernels take it)
            const long long n = a.nfft;
            if (!a.blue && n >= 64 && n <= 4096 && (n & (n - 1)) == 0) {
                const int E = (prec == P3_F32 && n >= 512 && n <= 2048) ? 32 : 16;
                const bool half = a.op == p3::OP_R2C_HALF || a.op == p3::OP_C2R_HALF;
                pd.twr = row_tw_table(T, n, E, half ? 2 * n : n) + 1;
            }
        } else {
            a.tpl = 1;
            a.nfft = a.n_in;  // slots per line; no FFT passes
            a.npass = 0;
        }
        tile_setup(a, P->csize, flags);
        Stage s;
        s.a = a; s.src = src; s.dst = dst; s.name = name; s.bytes = bytes;
        s.fused = false;
        P->st[dir].push_back(s);
        pend[dir].push_back(pd);
    };

    // ---- forward: X r2c, Y c2c, Z c2c / DCT-I / re-orientation ----------
    {
        const bool half = nx % 2 == 0;
        const int nfft = half ? nx / 2 : nx;
        StageArgs a = half ? base_args(p3::OP_R2C_HALF, nx, (int)H, nfft, -1, NY * NZ, rows(NY * NZ, RP),
                                       rows(NY * NZ, H))
                           : pair_args(p3::OP_R2C_PAIR, nx, (int)H, -1, rows(NY * NZ, RP), rows(NY * NZ, H));
        push(0, a, BUF_IN, zyx ? BUF_WS : BUF_OUT, "x_r2c", creal + ccplx, half ? nx : nx);
        const int work = zyx ? BUF_WS : BUF_OUT;
        if (ttype[1] == P3_FFT && ny > 1) {
            a = base_args(p3::OP_C2C, ny, ny, ny, -1, H * NZ, mapY, mapY);
            push(0, a, work, work, "y_c2c", 2 * ccplx, ny);
        }
        const LineMap zout = zyx ? mapZzyx : mapZxyz;
        if (ttype[2] == P3_FFT && nz > 1) {
            a = base_args(p3::OP_C2C, nz, nz, nz, -1, H * NY, mapZxyz, zout);
            push(0, a, work, BUF_OUT, zyx ? "z_c2c_zyx" : "z_c2c", 2 * ccplx, nz);
        } else if (ttype[2] == P3_CHEB) {
            a = base_args(p3::OP_DCT1, nz, nz, 2 * (nz - 1), -1, H * NY, mapZxyz, zout);
            push(0, a, work, BUF_OUT, zyx ? "z_dct1_zyx" : "z_dct1", 2 * ccplx, 2 * (nz - 1));
        } else if (ttype[2] == P3_SINE) {
            a = base_args(p3::OP_DST1, nz, nz, 2 * (nz + 1), -1, H * NY, mapZxyz, zout);
            push(0, a, work, BUF_OUT, zyx ? "z_dst1_zyx" : "z_dst1", 2 * ccplx, 2 * (nz + 1));
        } else if (zyx) {
            a = base_args(p3::OP_COPY, nz, nz, 1, -1, H * NY, mapZxyz, zout);
            push(0, a, work, BUF_OUT, "z_copy_zyx", 2 * ccplx, 1);
        }
    }
    // ---- inverse: Z, Y, X c2r -------------------------------------------
    // The work buffer is the workspace, or with padded real rows the output
    // itself (it holds H*Ny*Nz complex values), so the input stays untouched
    // out of place and everything runs in place when in == out.
    const int WORK = padded ? BUF_OUT : BUF_WS;
    {
        int cur = BUF_IN;
        const LineMap zin = zyx ? mapZzyx : mapZxyz;
        StageArgs a;
        if (ttype[2] == P3_FFT && nz > 1) {
            a = base_args(p3::OP_C2C, nz, nz, nz, +1, H * NY, zin, mapZxyz);
            push(1, a, cur, WORK, zyx ? "z_c2c_zyx_inv" : "z_c2c_inv", 2 * ccplx, nz);
            cur = WORK;
        } else if (ttype[2] == P3_CHEB) {
            a = base_args(p3::OP_DCT1, nz, nz, 2 * (nz - 1), +1, H * NY, zin, mapZxyz);
            push(1, a, cur, WORK, zyx ? "z_dct1_zyx_inv" : "z_dct1_inv", 2 * ccplx, 2 * (nz - 1));
            cur = WORK;
        } else if (ttype[2] == P3_SINE) {
            // DST-I is its own inverse up to 2(Nz+1): same sign both ways
            a = base_args(p3::OP_DST1, nz, nz, 2 * (nz + 1), -1, H * NY, zin, mapZxyz);
            push(1, a, cur, WORK, zyx ? "z_dst1_zyx_inv" : "z_dst1_inv", 2 * ccplx, 2 * (nz + 1));
            cur = WORK;
        } else if (zyx) {
            a = base_args(p3::OP_COPY, nz, nz, 1, +1, H * NY, zin, mapZxyz);
            push(1, a, cur, WORK, "z_copy_zyx_inv", 2 * ccplx, 1);
            cur = WORK;
        }
        if (ttype[1] == P3_FFT && ny > 1) {
            a = base_args(p3::OP_C2C, ny, ny, ny, +1, H * NZ, mapY, mapY);
            push(1, a, cur, WORK, "y_c2c_inv", 2 * ccplx, ny);
            cur = WORK;
        }
        const bool half = nx % 2 == 0;
        const int nfft = half ? nx / 2 : nx;
        a = half ? base_args(p3::OP_C2R_HALF, (int)H, nfft, nfft, +1, NY * NZ, rows(NY * NZ, H), rows(NY * NZ, RP))
                 : pair_args(p3::OP_C2R_PAIR, (int)H, nx, +1, rows(NY * NZ, H), rows(NY * NZ, RP));
        push(1, a, cur, BUF_OUT, "x_c2r", creal + ccplx, nx);
    }
    // ---- inverse with a user Z hook (EMPTY third dimension) ---------------
    // The hook runs on a copy of the input in the work buffer (XYZ order),
    // so the input stays untouched; then the inverse Y and X stages.
    if (ttype[2] == P3_EMPTY) {
        const LineMap zin = zyx ? mapZzyx : mapZxyz;
        StageArgs a = base_args(p3::OP_COPY, nz, nz, 1, +1, H * NY, zin, mapZxyz);
        push(2, a, BUF_IN, WORK, zyx ? "z_copy_zyx_inv" : "z_copy_inv", 2 * ccplx, 1);
        if (ttype[1] == P3_FFT && ny > 1) {
            a = base_args(p3::OP_C2C, ny, ny, ny, +1, H * NZ, mapY, mapY);
            push(2, a, WORK, WORK, "y_c2c_inv", 2 * ccplx, ny);
        }
        const bool half = nx % 2 == 0;
        const int nfft = half ? nx / 2 : nx;
        a = half ? base_args(p3::OP_C2R_HALF, (int)H, nfft, nfft, +1, NY * NZ, rows(NY * NZ, H), rows(NY * NZ, RP))
                 : pair_args(p3::OP_C2R_PAIR, (int)H, nx, +1, rows(NY * NZ, H), rows(NY * NZ, RP));
        push(2, a, WORK, BUF_OUT, "x_c2r", creal + ccplx, nx);
    }
    if (rc != P3_OK) {
        delete P;
        return rc;
    }
    // the stage lists before fusion (separate X and Y launches, plain
    // planes): the autotuner's other candidate
    std::vector<Stage> unfused[3] = {P->st[0], P->st[1], P->st[2]};
    // ---- plane-fused X + Y launches ----------------------------------------
    // fwd: stages 0 (X, src -> work) and 1 (Y in place on work); inverse and
    // hook-mode inverse: stages 1 (Y in place on work) and 2 (X, work -> out)
    int fuse_at[3] = {-1, -1, -1};
    p3::PlaneArgs fcfg[3];
    const bool may_fuse = !(flags & (P3_FLAG_NO_FUSE | P3_FLAG_PADDED_REAL)) && ttype[1] == P3_FFT && ny > 1;
    for (int d = 0; may_fuse && d < 3; ++d) {
        const int i = d == 0 ? 0 : 1;
        auto& v = P->st[d];
        if ((int)v.size() < i + 2) continue;
        const Stage& s0 = v[i];
        const Stage& s1 = v[i + 1];
        const Stage& sx = d == 0 ? s0 : s1;
        const Stage& sy = d == 0 ? s1 : s0;
        if (sy.src != sy.dst || (d == 0 ? sx.dst != sy.src : sx.src != sy.dst)) continue;
        // with the ZYX layout the planes between the stages live only in the
        // workspace, so they are stored transposed ([x][y]: contiguous Y
        // lines); the Z stage of the direction addresses them that way
        const bool tp = zyx && d < 2 && ttype[2] != P3_EMPTY;
        if (!p3::fused_configure(fcfg[d], sx.a, sy.a, d == 0 ? 0 : 1, P->csize, tp)) continue;
        fuse_at[d] = i;
        if (tp) {
            const LineMap ws_lines = LineMap{H * NY, 0, 1, H * NY};  // line x * Ny + y of planes [x][y]
            const LineMap zyx_lines = LineMap{H * NY, 0, NZ, 1};    // the same line in ZYX order
            Stage& z = d == 0 ? v[2] : v[0];
            if (d == 0) {
                z.a.in = ws_lines;
                z.a.out = zyx_lines;
            } else {
                z.a.in = zyx_lines;
                z.a.out = ws_lines;
            }
            // same kernel kind; the new maps can admit a TMA-fed variant
            if (z.a.kern != p3::KIND_GENERIC) p3::pow2_configure(z.a, P->csize, !(flags & P3_FLAG_NO_TMA));
        }
    }
    const bool any_fused = fuse_at[0] >= 0 || fuse_at[1] >= 0 || fuse_at[2] >= 0;
    bool need_ws = false;
    for (int d = 0; d < 3; ++d)
        for (auto& s : P->st[d])
            if (s.src == BUF_WS || s.dst == BUF_WS) need_ws = true;
    const size_t cbytes = (size_t)P->csize * (size_t)H * (size_t)NY * (size_t)NZ;
    P->ctr_off = need_ws ? (cbytes + 255) / 256 * 256 : 0;
    P->ws_bytes = (need_ws ? cbytes : 0);
    if (any_fused) P->ws_bytes = P->ctr_off + (sizeof(unsigned) * (size_t)(NZ + 1) + 255) / 256 * 256;

    // ---- device tables ------------------------------------------------------
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return P3_ERR_CUDA;
    }
    if (p3::prepare_kernels() != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return P3_ERR_CUDA;
    }
    const size_t nvals = T.vals.size();
    const size_t bytes = nvals * P->csize;
    if (bytes) {
        std::vector<unsigned char> host(bytes);
        for (size_t i = 0; i < nvals; ++i) {
            if (prec == P3_F32) {
                float v[2] = {(float)T.vals[i].real(), (float)T.vals[i].imag()};
                memcpy(&host[i * 8], v, 8);
            } else {
                double v[2] = {T.vals[i].real(), T.vals[i].imag()};
                memcpy(&host[i * 16], v, 16);
            }
        }
        cudaError_t ce = cudaMalloc(&P->dtab, bytes);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            delete P;
            return ce == cudaErrorMemoryAllocation ? P3_ERR_NOMEM : P3_ERR_CUDA;
        }
        ce = cudaMemcpy(P->dtab, host.data(), bytes, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            cudaFree(P->dtab);
            delete P;
            return P3_ERR_CUDA;
        }
    }
    auto resolve = [&](size_t off) -> const void* {
        return off ? (const void*)((const unsigned char*)P->dtab + (off - 1) * P->csize) : NULL;
    };
    for (int d = 0; d < 3; ++d) {
        for (size_t i = 0; i < P->st[d].size(); ++i) {
            StageArgs& a = P->st[d][i].a;
            const Pending& pd = pend[d][i];
            a.tw = resolve(pd.tw);
            a.tw2 = resolve(pd.tw2);
            a.chirp = resolve(pd.chirp);
            a.bhat = resolve(pd.bhat);
            a.twm = resolve(pd.twm);
            a.twr = resolve(pd.twr);
            StageArgs& b = unfused[d][i].a;
            b.twr = a.twr;
            b.tw = a.tw;
            b.tw2 = a.tw2;
            b.chirp = a.chirp;
            b.bhat = a.bhat;
            b.twm = a.twm;
        }
    }
    for (int d = 0; d < 3; ++d) {
        const int i = fuse_at[d];
        if (i < 0) continue;
        auto& v = P->st[d];
        Stage& sx = d == 0 ? v[i] : v[i + 1];
        Stage& sy = d == 0 ? v[i + 1] : v[i];
        p3::PlaneArgs f = fcfg[d];
        f.x = sx.a;
        f.y = sy.a;
        f.y.nlines = H;  // one plane's Y lines: L = x, in place
        f.y.in = LineMap{H, 0, 1, H};
        f.y.out = f.y.in;
        f.nplanes = nz;
        f.rows = ny;
        f.yoff = NY * H;
        f.xt = (int)((NY + f.bx - 1) / f.bx);
        f.yt = (int)((H + f.by - 1) / f.by);
        // lag: about three (forward) or one and a half (inverse) grid-fulls
        // of tickets between a plane's last producer and its first consumer
        // (measured best at 1024^3), capped at the number of planes that fit
        // in 48 MB of the 129 MB L2 (2048^3: lag 2, measured within 4 % of the
        // best lag)
        {
            const long long per = f.xt + f.yt;
            const long long span = d == 0 ? 3LL * f.grid : 3LL * f.grid / 2;
            long long lag = (span + per - 1) / per + 1;
            const long long plane_bytes = (long long)P->csize * NY * H;
            const long long cap = (48LL << 20) / (plane_bytes > 0 ? plane_bytes : 1);
            if (lag > cap) lag = cap;
            if (lag > nz) lag = nz;
            if (lag < 1) lag = 1;
            f.lag = (int)lag;
        }
        P->fused_lag_default[d] = f.lag;
        Stage m = sx;
        m.src = d == 0 ? sx.src : sy.src;
        m.dst = sx.dst;
        m.name = d == 0 ? "xy_fused" : "yx_fused_inv";
        m.bytes = creal + ccplx;
        m.fused = true;
        m.f = f;
        v.erase(v.begin() + i, v.begin() + i + 2);
        v.insert(v.begin() + i, m);
    }
    {  // the plan's device status word (bounded waits of fused and TMA kernels)
        cudaError_t ce = cudaMalloc(&P->derr, 256);
        if (ce == cudaSuccess) ce = cudaMemset(P->derr, 0, 256);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            if (P->dtab) cudaFree(P->dtab);
            if (P->derr) cudaFree(P->derr);
            delete P;
            return P3_ERR_NOMEM;
        }
    }
    P->st_unfused[0] = unfused[0];
    P->st_unfused[1] = unfused[1];
    // ---- autotuning (P3_FLAG_TUNE) -------------------------------------------
    std::string tuned;
    if (flags & P3_FLAG_TUNE) {
        rc = tune_generic(P, tuned);
        if (rc != P3_OK) {
            if (P->dtab) cudaFree(P->dtab);
            if (P->derr) cudaFree(P->derr);
            cudaGetLastError();
            delete P;
            return rc;
        }
    }
    // the batched persistent launch starts from the tuned radix orders too
    for (int d = 0; d < 2; ++d) {
        bool fused = false;
        for (const Stage& s : P->st[d]) fused = fused || s.fused;
        if (!fused) P->st_unfused[d] = P->st[d];
    }
    if ((flags & P3_FLAG_TUNE) && any_fused) {
        rc = tune(P, unfused, tuned);
        if (rc != P3_OK) {
            if (P->dtab) cudaFree(P->dtab);
            if (P->derr) cudaFree(P->derr);
            cudaGetLastError();
            delete P;
            return rc;
        }
    }
    // ---- description ----------------------------------------------------------
    char line[512];
    for (int d = 0; d < 2; ++d) {
        std::string groups;  // one timing group per stage launch, in order
        for (auto& s : P->st[d]) groups += (groups.empty() ? "" : ",") + std::string(s.name);
        snprintf(line, sizeof(line), "%s groups=%s\n", d == 0 ? "fwd" : "bwd", groups.c_str());
        P->desc += line;
        for (auto& s : P->st[d]) {
            const StageArgs& a = s.a;
            if (s.fused) {
                const p3::PlaneArgs& f = s.f;
                snprintf(line, sizeof(line),
                         "%s %s kernel=plane_fused x_nfft=%d y_nfft=%d planes=%d x_tiles=%d y_tiles=%d lag=%d "
                         "persistent_ctas=%d threads=%d smem=%zu bytes=%.0f\n",
                         d == 0 ? "fwd" : "bwd", s.name, f.kx, f.ky, f.nplanes, f.xt, f.yt, f.lag, f.grid, f.nt, f.smem,
                         s.bytes);
                P->desc += line;
                continue;
            }
            std::string rs;
            if (a.kern != p3::KIND_GENERIC) {
                // power-of-two kernels: radix E = nfft / tpl while it divides, then the rest
                const int E = a.nfft / a.tpl;
                int n = a.nfft;
                while (n % E == 0 && n >= E) {
                    rs += std::to_string(E) + "x";
                    n /= E;
                }
                if (n > 1) rs += std::to_string(n) + "x";
                rs.pop_back();
            } else {
                const int np = a.blue ? a.mpass : a.npass;
                for (int i = 0; i < np; ++i) {
                    rs += std::to_string(a.blue ? a.mrad[i] : a.rad[i]);
                    if (i + 1 < np) rs += "x";
                }
            }
            if (rs.empty()) rs = "-";
            snprintf(line, sizeof(line),
                     "%s %s kernel=%s op=%s nfft=%d%s radices=%s lines=%lld B=%d LDB=%d tpl=%d threads=%d "
                     "smem=%zu bytes=%.0f\n",
                     d == 0 ? "fwd" : "bwd", s.name, kern_name(a.kern, a.tc, a.tma), op_name(a.op), a.nfft,
                     a.blue ? (" bluestein_m=" + std::to_string(a.m)).c_str() : "", rs.c_str(), a.nlines, a.B,
                     a.LDB, a.tpl, a.threads, a.smem, s.bytes);
            P->desc += line;
        }
    }
    if (!tuned.empty()) P->desc += tuned;
    if (!P->st[2].empty()) {
        std::string names;
        for (auto& s : P->st[2]) names += (names.empty() ? "" : ",") + std::string(s.name);
        snprintf(line, sizeof(line), "z_hook fwd: after %s; bwd: after %s, then %s\n",
                 P->st[0].empty() ? "-" : P->st[0].back().name, P->st[2][0].name, names.c_str());
        P->desc += line;
    }
    *out = P;
    return P3_OK;
}

p3_status p3_plan_destroy(p3_plan plan)
{
    if (!plan) return P3_OK;
    if (plan->dtab) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != plan->device) cudaSetDevice(plan->device);
        cudaFree(plan->dtab);
        if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
        cudaGetLastError();
    }
    if (plan->derr) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != plan->device) cudaSetDevice(plan->device);
        cudaFree(plan->derr);
        if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
        cudaGetLastError();
    }
    delete plan;
    return P3_OK;
}

// The Z lines of the array the hook sees: ZYX output, Z contiguous; XYZ
// (forward output or the inverse work copy), Z strided by H * Ny.
static int call_hook(p3_plan P, int dir, void* data, void* stream)
{
    const long long H = P->H, NY = P->ny, NZ = P->nz;
    const bool zyx = dir == 0 && P->layout == P3_LAYOUT_ZYX;
    return P->hook(data, P->nz, H * NY, zyx ? NZ : 1, zyx ? 1 : H * NY, dir, stream, P->hook_user);
}

// The argument checks of a call (Sect. 3.2 semantics: const input, caller
// buffers), without launching: NULL / misaligned / overlapping buffers, a
// missing workspace, the wrong device.  uses_ws: whether `stages` use it.
static p3_status check_call(p3_plan P, int dir, const void* in, void* out, void* ws,
                            const std::vector<Stage>& stages)
{
    if (!P || !in || !out) return P3_ERR_INVALID;
    if (!aligned16(in) || !aligned16(out) || (ws && !aligned16(ws))) return P3_ERR_INVALID;
    if (in == out && !P->padded) return P3_ERR_UNSUPPORTED;
    const size_t rowr = P->padded ? 2 * (size_t)P->H : (size_t)P->nx;
    const size_t nreal = rowr * P->ny * P->nz * (P->csize / 2);
    const size_t ncplx = (size_t)P->H * P->ny * P->nz * P->csize;
    const size_t nin = dir == 0 ? nreal : ncplx, nout = dir == 0 ? ncplx : nreal;
    if (in != out && overlap(in, nin, out, nout)) return P3_ERR_INVALID;
    bool uses_ws = false;
    for (auto& s : stages)
        if (s.src == BUF_WS || s.dst == BUF_WS || s.fused) uses_ws = true;
    if (uses_ws) {
        if (!ws) return P3_ERR_WORKSPACE;
        if (overlap(ws, P->ws_bytes, in, nin) || overlap(ws, P->ws_bytes, out, nout)) return P3_ERR_INVALID;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (cur != P->device) return P3_ERR_INVALID;
    return P3_OK;
}

static p3_status run(p3_plan P, int dir, const void* in, void* out, void* ws, void* stream)
{
    if (!P || !in || !out) return P3_ERR_INVALID;
    // a Z hook replaces the empty third-dimension transform: forward, it
    // runs after the last stage; inverse, after the copy of the input into
    // the work buffer that starts the hook-mode stage list
    const p3_z_hook hook = P->hook;
    const std::vector<Stage>& stages = (dir == 1 && hook) ? P->st[2] : P->st[dir];
    const size_t hook_after = hook ? (dir == 0 ? stages.size() : 1) : 0;
    const p3_status chk = check_call(P, dir, in, out, ws, stages);
    if (chk != P3_OK) return chk;
    cudaStream_t s = (cudaStream_t)stream;
    void* const bufs[3] = {const_cast<void*>(in), out, ws};
    cudaEvent_t* ev = P->timing ? (cudaEvent_t*)&P->events[dir * 4] : NULL;
    if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return P3_ERR_CUDA;
    int i = 0;
    for (auto& st : stages) {
        StageArgs a = st.a;
        a.src = bufs[st.src];
        a.dst = bufs[st.dst];
        a.err = P->derr;
        a.spin = P->spin_limit / 2 > 0 ? P->spin_limit / 2 : 1;
        a.wait_extra = P->wait_extra ? 1 : 0;
        cudaError_t e;
        if (st.fused) {
            p3::PlaneArgs f = st.f;
            f.x.src = bufs[st.src];
            f.x.dst = bufs[st.dst];
            void* yb = bufs[dir == 0 ? st.dst : st.src];
            f.y.src = yb;
            f.y.dst = yb;
            f.ctr = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ws) + P->ctr_off);
            f.err = P->derr;
            f.spin_limit = P->spin_limit;
            f.extra = P->wait_extra;
            e = p3::fused_launch(f, s);
        } else {
            e = a.tma == 1 ? p3::pow2_encode_tma(a) : cudaSuccess;
            if (e == cudaSuccess) e = P->prec == P3_F32 ? p3::launch_stage_f32(a, s) : p3::launch_stage_f64(a, s);
        }
        if (e != cudaSuccess) return P3_ERR_CUDA;
        ++i;
        if (hook && (size_t)i == hook_after && call_hook(P, dir, a.dst, stream) != 0) return P3_ERR_HOOK;
        if (ev && i <= 3 && cudaEventRecord(ev[i], s) != cudaSuccess) return P3_ERR_CUDA;
    }
    if (hook && stages.empty() && call_hook(P, dir, out, stream) != 0) return P3_ERR_HOOK;
    if (ev)
        for (int k = i + 1; k <= 3; ++k)
            if (cudaEventRecord(ev[k], s) != cudaSuccess) return P3_ERR_CUDA;
    return P3_OK;
}

p3_status p3_ftran_r2c(p3_plan plan, const void* in_real, void* out_cplx, void* workspace, void* stream)
{
    return run(plan, 0, in_real, out_cplx, workspace, stream);
}

p3_status p3_btran_c2r(p3_plan plan, const void* in_cplx, void* out_real, void* workspace, void* stream)
{
    return run(plan, 1, in_cplx, out_real, workspace, stream);
}

p3_status p3_plan_get_dims(p3_plan plan, int in_dims[3], int out_dims[3])
{
    if (!plan || !in_dims || !out_dims) return P3_ERR_INVALID;
    in_dims[0] = plan->nx; in_dims[1] = plan->ny; in_dims[2] = plan->nz;
    if (plan->layout == P3_LAYOUT_XYZ) {
        out_dims[0] = plan->H; out_dims[1] = plan->ny; out_dims[2] = plan->nz;
    } else {
        out_dims[0] = plan->nz; out_dims[1] = plan->ny; out_dims[2] = plan->H;
    }
    return P3_OK;
}

p3_status p3_plan_workspace_bytes(p3_plan plan, size_t* bytes)
{
    if (!plan || !bytes) return P3_ERR_INVALID;
    *bytes = plan->ws_bytes;
    return P3_OK;
}

p3_status p3_plan_scale(p3_plan plan, double* scale)
{
    if (!plan || !scale) return P3_ERR_INVALID;
    *scale = plan->scale;
    return P3_OK;
}

p3_status p3_plan_set_stage_events(p3_plan plan, void* const* events, int n_events)
{
    if (!plan) return P3_ERR_INVALID;
    if (!events) {
        plan->timing = false;
        memset(plan->events, 0, sizeof(plan->events));
        return P3_OK;
    }
    if (n_events != 8) return P3_ERR_INVALID;
    for (int i = 0; i < 8; ++i)
        if (!events[i]) return P3_ERR_INVALID;
    for (int i = 0; i < 8; ++i) plan->events[i] = events[i];
    plan->timing = true;
    return P3_OK;
}

p3_status p3_plan_describe(p3_plan plan, char* buf, size_t len)
{
    if (!plan || !buf) return P3_ERR_INVALID;
    if (len == 0) return P3_OK;
    const size_t n = plan->desc.size() < len - 1 ? plan->desc.size() : len - 1;
    memcpy(buf, plan->desc.data(), n);
    buf[n] = 0;
    return P3_OK;
}

p3_status p3_plan_factor(int n, p3_precision prec, int* radices, int cap, int* npass)
{
    if (n < 2 || !radices || !npass || cap < 1 || (prec != P3_F32 && prec != P3_F64)) return P3_ERR_INVALID;
    const bool composite = prec == P3_F32 && P3_GEN_COMPOSITE;
    std::vector<int> rad;
    if (!factor(n, rad, composite) || !radices_supported(rad, composite)) return P3_ERR_UNSUPPORTED;
    if ((int)rad.size() > cap) return P3_ERR_UNSUPPORTED;
    for (size_t i = 0; i < rad.size(); ++i) radices[i] = rad[i];
    *npass = (int)rad.size();
    return P3_OK;
}

p3_status p3_plan_launches(p3_plan plan, int dir, int* launches)
{
    if (!plan || !launches || (dir != 0 && dir != 1)) return P3_ERR_INVALID;
    *launches = (int)plan->st[dir == 1 && plan->hook ? 2 : dir].size();
    return P3_OK;
}

p3_status p3_plan_wait_status(p3_plan plan)
{
    if (!plan) return P3_ERR_INVALID;
    if (!plan->derr) return P3_OK;
    unsigned v = 0;
    if (cudaMemcpy(&v, plan->derr, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (!v) return P3_OK;
    if (cudaMemset(plan->derr, 0, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    return P3_ERR_TIMEOUT;
}

p3_status p3_plan_wait_flags(p3_plan plan, unsigned* flags)
{
    if (!plan || !flags) return P3_ERR_INVALID;
    *flags = 0;
    if (!plan->derr) return P3_OK;
    if (cudaMemcpy(flags, plan->derr, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (*flags && cudaMemset(plan->derr, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    return P3_OK;
}

p3_status p3_plan_set_fused_lag(p3_plan plan, int lag)
{
    if (!plan || lag < 0) return P3_ERR_INVALID;
    for (int d = 0; d < 3; ++d)
        for (auto& s : plan->st[d])
            if (s.fused) s.f.lag = lag == 0 ? plan->fused_lag_default[d] : (lag < s.f.nplanes ? lag : s.f.nplanes);
    return P3_OK;
}

p3_status p3_plan_set_wait_limits(p3_plan plan, unsigned spin_limit, unsigned extra)
{
    if (!plan || spin_limit == 0) return P3_ERR_INVALID;
    plan->spin_limit = spin_limit;
    plan->wait_extra = extra;
    return P3_OK;
}

p3_status p3_plan_set_z_hook(p3_plan plan, p3_z_hook fn, void* user)
{
    if (!plan) return P3_ERR_INVALID;
    if (plan->tt[2] != P3_EMPTY) return P3_ERR_INVALID;
    plan->hook = fn;
    plan->hook_user = fn ? user : NULL;
    return P3_OK;
}

}  // extern "C"

#ifndef P3_BATCH_SMEM
#define P3_BATCH_SMEM (54 * 1024)
#endif

namespace p3 {
p3_status run_direction(p3_plan plan, int dir, const void* in, void* out, void* ws, void* stream)
{
    return run(plan, dir, in, out, ws, stream);
}
p3_status generic_stages(p3_plan P, int dir, std::vector<GenericStage>& out)
{
    out.clear();
    if (!P || (dir != 0 && dir != 1)) return P3_ERR_INVALID;
    for (const Stage& s : P->st_unfused[dir]) {
        GenericStage g;
        g.a = s.a;
        if (g.a.op != OP_COPY) {
            const int len = g.a.blue ? g.a.m : g.a.nfft;
            if (len > 1) {
                const int* r = g.a.blue ? g.a.mrad : g.a.rad;
                const int np = g.a.blue ? g.a.mpass : g.a.npass;
                g.a.tpl = threads_per_line(len, std::vector<int>(r, r + np));
            } else {
                g.a.tpl = 1;
            }
        }
        // tiles of at most P3_BATCH_SMEM bytes, so that the batched kernel
        // keeps its resident CTAs whatever stage it runs
        generic_tile_setup(g.a, P->csize, P3_BATCH_SMEM, p3::kMaxThreads);
        g.src = s.src;
        g.dst = s.dst;
        out.push_back(g);
    }
    return P3_OK;
}
p3_status check_generic_call(p3_plan P, int dir, const void* in, void* out, void* ws)
{
    if (!P || (dir != 0 && dir != 1)) return P3_ERR_INVALID;
    return check_call(P, dir, in, out, ws, P->st_unfused[dir]);
}
bool plan_batchable(p3_plan P) { return P && P->prec == P3_F32 && !P->hook; }
size_t plan_workspace(p3_plan plan) { return plan ? plan->ws_bytes : 0; }
double plan_work(p3_plan plan) { return plan ? (double)plan->nx * plan->ny * plan->nz : 0.0; }
int plan_device(p3_plan plan) { return plan ? plan->device : -1; }
}  // namespace p3
