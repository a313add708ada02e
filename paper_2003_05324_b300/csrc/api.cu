// C ABI of libgeo (declared in include/geo.h): argument checking, workspace
// layout, and the host-side sequencing of the device work.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "geo_internal.cuh"
#include "dag.cuh"
#include "lp_gemm.cuh"

namespace geo {

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// meta buffer: off[p*p] int64 | slot[p*p] int32 | status[16] + tickets[2p] int32 |
// scal doubles | (tensor-core mode) scheduler counters | per scheduling variant
// (0: in-band updates on the tensor cores, 1: on the FP64 pipe, 2: the DST
// approximation): CUDA-core tasks, bulk tasks, solve ends, tensor targets
constexpr int N_VARIANTS = 3;
struct MetaOffsets {
    size_t off, slot, far, status, scal, sched_ctr, total;
    size_t sched_g2[N_VARIANTS], sched_bulk[N_VARIANTS], sched_end[N_VARIANTS], sched_tct[N_VARIANTS],
        sched_y[N_VARIANTS];
    SchedGeom geom[N_VARIANTS];
    bool dag;
};

static MetaOffsets meta_offsets(int p, int nb, int band, int lp_mode, int pp) {
    MetaOffsets m;
    size_t b = 0;
    m.off = b;
    b = align256(b + sizeof(long long) * (size_t)p * p);
    m.slot = b;
    b = align256(b + sizeof(int) * (size_t)p * p);
    m.far = b;
    b = align256(b + (size_t)p * p);
    m.status = b;
    b = align256(b + sizeof(int) * ((size_t)ST_WORDS + 2 * (size_t)p));
    m.scal = b;
    b = align256(b + sizeof(double) * ((size_t)2 * p + 8 + (size_t)p * nb));
    m.dag = (lp_mode == GEO_LP_SPLIT_BF16);
    m.sched_ctr = b;
    for (int v = 0; v < N_VARIANTS; ++v) {
        m.geom[v] = sched_geom(p, nb, band, pp, v != 1, v == 2);
        m.sched_g2[v] = m.sched_bulk[v] = m.sched_end[v] = m.sched_tct[v] = m.sched_y[v] = b;
    }
    if (m.dag) {
        b = align256(b + sizeof(int) * (size_t)m.geom[0].n_counters);   // the same counters for every variant
        for (int v = 0; v < N_VARIANTS; ++v) {
            const SchedGeom& g = m.geom[v];
            m.sched_g2[v] = b;
            b = align256(b + sizeof(G2Task) * (size_t)g.n_prio);
            m.sched_bulk[v] = b;
            b = align256(b + sizeof(G2Task) * (size_t)std::max(g.n_bulk, 1LL));
            m.sched_end[v] = b;
            b = align256(b + sizeof(int) * (size_t)p);
            m.sched_tct[v] = b;
            b = align256(b + sizeof(int4) * (size_t)std::max(g.n_tct, 1LL));
            m.sched_y[v] = b;
            b = align256(b + sizeof(G2Task) * (size_t)std::max(g.n_y, 1LL));
        }
    }
    m.total = b;
    return m;
}

static MetaOffsets meta_offsets(const geo_layout& g) { return meta_offsets(g.p, g.nb, g.band, g.lp_mode, g.pp); }

// ---- instrumentation ------------------------------------------------------
static std::atomic<unsigned long long> g_launches{0};
static bool g_prof = false;
struct ProfSlot {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> open;   // recorded, not yet summed
    std::vector<cudaEvent_t> pool;
    double ms = 0.0;
    long long launches = 0;
};
static ProfSlot g_slots[6];
static std::mutex g_prof_mu;

void count_launch(int n) { g_launches += (unsigned long long)n; }
bool prof_on() { return g_prof; }

static cudaEvent_t take_event(ProfSlot& sl) {
    if (!sl.pool.empty()) {
        cudaEvent_t e = sl.pool.back();
        sl.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(int kind, cudaStream_t s) {
    if (!g_prof) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfSlot& sl = g_slots[kind];
    cudaEvent_t e0 = take_event(sl), e1 = take_event(sl);
    cudaEventRecord(e0, s);
    sl.open.push_back({e0, e1});
}

void prof_end(int kind, cudaStream_t s) {
    if (!g_prof) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfSlot& sl = g_slots[kind];
    if (sl.open.empty()) return;
    cudaEventRecord(sl.open.back().second, s);
    sl.launches += 1;
}

static void prof_collect(ProfSlot& sl) {
    for (auto& pr : sl.open) {
        float ms = 0.0f;
        cudaEventSynchronize(pr.second);
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) sl.ms += ms;
        sl.pool.push_back(pr.first);
        sl.pool.push_back(pr.second);
    }
    sl.open.clear();
}

Layout make_layout(const geo_tiles* t) {
    Layout L;
    const geo_layout& g = t->lay;
    L.n = g.n;
    L.nb = g.nb;
    L.p = g.p;
    L.band = g.band;
    L.pp = g.pp;
    L.lp_mode = g.lp_mode;
    L.flags = t->flags;
    L.dp = t->d_dp;
    L.sp = t->d_sp;
    MetaOffsets mo = meta_offsets(g);
    char* base = (char*)t->d_meta;
    L.off = (const long long*)(base + mo.off);
    L.slot = (const int*)(base + mo.slot);
    L.status = (int*)(base + mo.status);
    L.tickets = L.status + ST_WORDS;
    L.scal = (double*)(base + mo.scal);
    L.far = t->far_products ? (const unsigned char*)(base + mo.far) : nullptr;
    L.far_products = t->far_products;
    L.planes = (__nv_bfloat16*)t->d_planes;
    L.npl = planes_per_slot(g.band, g.p);
    L.rexp = t->d_planes ? (int*)((char*)t->d_planes + align256((size_t)L.npl * g.pp * g.pp *
                                                                sizeof(__nv_bfloat16) * (size_t)g.n_slots))
                         : nullptr;
    return L;
}

}  // namespace geo

using namespace geo;

extern "C" {

int geo_morton_order(const double* x, const double* y, int n, int* perm) {
    if (!x) return -1;
    if (!y) return -2;
    if (n < 0) return -3;
    if (!perm && n > 0) return -4;
    std::vector<std::pair<unsigned long long, int>> kv((size_t)n);
    for (int idx = 0; idx < n; ++idx) {
        long long qx = (long long)floor(x[idx] * 65536.0), qy = (long long)floor(y[idx] * 65536.0);
        qx = std::min(std::max(qx, 0LL), 65535LL);
        qy = std::min(std::max(qy, 0LL), 65535LL);
        unsigned long long key = 0;
        for (int b = 0; b < 16; ++b) {
            key |= (unsigned long long)((qx >> b) & 1) << (2 * b);
            key |= (unsigned long long)((qy >> b) & 1) << (2 * b + 1);
        }
        kv[(size_t)idx] = {key, idx};
    }
    std::sort(kv.begin(), kv.end());   // (key, index) pairs: ties keep the original order
    for (int idx = 0; idx < n; ++idx) perm[idx] = kv[(size_t)idx].second;
    return GEO_OK;
}

int geo_layout_init(int n, int nb, int band, int lp_mode, geo_layout* out) {
    if (n < 1) return -1;
    if (nb < 16 || nb > 768) return -2;
    if (band < 1) return -3;
    if (lp_mode != GEO_LP_SPLIT_BF16 && lp_mode != GEO_LP_FP32) return -4;
    if (!out) return -5;
    const int p = (n + nb - 1) / nb;
    if ((long long)p * (p + 1) / 2 > 65535) return -1;   // grid-y bound of the per-tile launches
    geo_layout g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.nb = nb;
    g.p = p;
    g.band = std::min(band, p);
    g.lp_mode = lp_mode;
    g.pp = (nb + 63) / 64 * 64;
    long long ndp = 0, nsp = 0;
    for (int j = 0; j < p; ++j)
        for (int i = j; i < p; ++i) (is_dp(i, j, g.band) ? ndp : nsp) += 1;
    g.n_dp_tiles = ndp;
    g.n_sp_tiles = nsp;
    g.n_slots = (long long)p * (p - 1) / 2;
    const size_t tile = (size_t)nb * nb;
    g.bytes_dp = align256(sizeof(double) * tile * (size_t)ndp);
    g.bytes_sp = align256(sizeof(float) * tile * (size_t)std::max(nsp, 1LL));
    // the slice planes of every panel tile (2 bytes per entry), then one int32
    // row exponent per plane row
    g.bytes_planes = (lp_mode == GEO_LP_SPLIT_BF16 && p > 1)
                         ? align256((size_t)planes_per_slot(g.band, p) * g.pp * g.pp * sizeof(__nv_bfloat16) *
                                    (size_t)g.n_slots) +
                               align256(sizeof(int) * (size_t)g.pp * (size_t)g.n_slots)
                         : 0;
    g.bytes_meta = meta_offsets(g).total;
    *out = g;
    return GEO_OK;
}

int geo_tiles_bind(geo_tiles* t, const geo_layout* lay, void* d_dp, void* d_sp, void* d_planes, void* d_meta,
                   void* stream) {
    if (!t) return -1;
    if (!lay || lay->p < 1) return -2;
    if (!d_dp) return -3;
    if (!d_sp) return -4;
    if (lay->bytes_planes > 0 && !d_planes) return -5;
    if (!d_meta) return -6;
    memset(t, 0, sizeof(*t));
    t->lay = *lay;
    t->d_dp = (double*)d_dp;
    t->d_sp = (float*)d_sp;
    t->d_planes = d_planes;
    t->d_meta = d_meta;
    const int p = lay->p, nb = lay->nb;
    const size_t tile = (size_t)nb * nb;
    MetaOffsets mo = meta_offsets(*lay);
    std::vector<char> host(mo.scal, 0);
    long long* off = (long long*)(host.data() + mo.off);
    int* slot = (int*)(host.data() + mo.slot);
    long long ndp = 0, nsp = 0;
    int ns = 0;
    for (int q = 0; q < p * p; ++q) {
        off[q] = -1;
        slot[q] = -1;
    }
    for (int j = 0; j < p; ++j)
        for (int i = j; i < p; ++i) {
            if (is_dp(i, j, lay->band)) off[i * p + j] = (long long)tile * ndp++;
            else off[i * p + j] = (long long)tile * nsp++;
            if (i > j) slot[i * p + j] = ns++;
        }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_meta, host.data(), mo.scal, cudaMemcpyHostToDevice, s);
    std::vector<G2Task> prio, bulk, yq;
    std::vector<int> trsm_end;
    std::vector<int4> tct;
    for (int v = 0; v < N_VARIANTS && !e && mo.dag; ++v) {
        sched_build(mo.geom[v], lay->band, prio, bulk, trsm_end, yq, tct);
        if (!prio.empty())
            e = cudaMemcpyAsync((char*)d_meta + mo.sched_g2[v], prio.data(), sizeof(G2Task) * prio.size(),
                                cudaMemcpyHostToDevice, s);
        if (!e && !bulk.empty())
            e = cudaMemcpyAsync((char*)d_meta + mo.sched_bulk[v], bulk.data(), sizeof(G2Task) * bulk.size(),
                                cudaMemcpyHostToDevice, s);
        if (!e)
            e = cudaMemcpyAsync((char*)d_meta + mo.sched_end[v], trsm_end.data(), sizeof(int) * trsm_end.size(),
                                cudaMemcpyHostToDevice, s);
        if (!e && !tct.empty())
            e = cudaMemcpyAsync((char*)d_meta + mo.sched_tct[v], tct.data(), sizeof(int4) * tct.size(),
                                cudaMemcpyHostToDevice, s);
        if (!e && !yq.empty())
            e = cudaMemcpyAsync((char*)d_meta + mo.sched_y[v], yq.data(), sizeof(G2Task) * yq.size(),
                                cudaMemcpyHostToDevice, s);
        if (!e) e = cudaStreamSynchronize(s);   // the host vectors are reused for the next variant
    }
    // padding rows of the slice planes are never written by the solves: zero them once
    if (!e && d_planes && lay->bytes_planes) e = cudaMemsetAsync(d_planes, 0, lay->bytes_planes, s);
    if (!e) e = cudaStreamSynchronize(s);
    cudaStream_t aux = nullptr;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    if (!e) e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&e2, cudaEventDisableTiming);
    if (e) return GEO_ERR_CUDA;
    t->aux_stream = aux;
    t->ev_fork = e1;
    t->ev_join = e2;
    if (lay->bytes_planes > 0 && prepare_lp_gemm(t, make_layout(t)) != 0) return GEO_ERR_CUDA;
    return GEO_OK;
}

int geo_tiles_release(geo_tiles* t) {
    if (!t) return -1;
    if (t->ev_fork) cudaEventDestroy((cudaEvent_t)t->ev_fork);
    if (t->ev_join) cudaEventDestroy((cudaEvent_t)t->ev_join);
    if (t->aux_stream) cudaStreamDestroy((cudaStream_t)t->aux_stream);
    t->ev_fork = t->ev_join = t->aux_stream = nullptr;
    return GEO_OK;
}

int geo_tiles_set_flags(geo_tiles* t, int flags) {
    if (!t) return -1;
    if (flags & ~(GEO_FLAG_FP64_OFFBAND_GEN | GEO_FLAG_STEPWISE | GEO_FLAG_FP64_DMMA | GEO_FLAG_DST |
                  GEO_FLAG_TEST_STALL))
        return -2;
    if ((flags & GEO_FLAG_DST) &&
        ((flags & (GEO_FLAG_STEPWISE | GEO_FLAG_FP64_DMMA)) || t->lay.lp_mode != GEO_LP_SPLIT_BF16))
        return -2;
    if ((flags & GEO_FLAG_STEPWISE) && t->far_products) return -2;   // the far tier runs in the persistent scheduler
    t->flags = flags;
    return GEO_OK;
}

int geo_tiles_set_timeout_ns(geo_tiles* t, long long ns) {
    if (!t) return -1;
    if (ns != 0 && (ns < 100000LL || ns > 1000000000000LL)) return -2;
    t->timeout_ns = ns;
    return GEO_OK;
}

int geo_tiles_set_far(geo_tiles* t, int far_band, const double* d_x, const double* d_y, double far_dist,
                      int products, void* stream) {
    if (!t || !t->d_meta) return -1;
    if (far_band < 0) return -2;
    if (far_dist > 0.0 && !d_x) return -3;
    if (far_dist > 0.0 && !d_y) return -4;
    if (!(far_dist == far_dist)) return -5;
    if (products != 1 && products != 3) return -6;
    if (far_band == 0 && !(far_dist > 0.0)) {   // tier off
        t->far_products = 0;
        return GEO_OK;
    }
    if (t->lay.lp_mode != GEO_LP_SPLIT_BF16 || !t->d_planes || (t->flags & GEO_FLAG_STEPWISE))
        return GEO_ERR_UNSUPPORTED;
    Layout L = make_layout(t);
    MetaOffsets mo = meta_offsets(t->lay);
    unsigned char* far = (unsigned char*)t->d_meta + mo.far;
    if (launch_far_map(L, far, far_band, d_x, d_y, far_dist, L.scal + 2 * L.p + 8, (cudaStream_t)stream))
        return GEO_ERR_CUDA;
    t->far_products = products;
    return GEO_OK;
}

int geo_tiles_set_trace(geo_tiles* t, void* d_trace, long long capacity) {
    if (!t) return -1;
    if (d_trace && capacity < 0) return -3;
    t->trace = d_trace;
    t->trace_cap = d_trace ? capacity : 0;
    return GEO_OK;
}

static int check_bound(const geo_tiles* t) { return (t && t->d_meta && t->d_dp && t->d_sp) ? 0 : 1; }

static int check_theta(const geo_theta& th) {
    return (th.sigma2 > 0 && th.beta > 0 && th.nu > 0 && th.nu <= 20 && th.nugget >= 0 && isfinite(th.sigma2) &&
            isfinite(th.beta))
               ? 0
               : 1;
}

int geo_matern_tiles(geo_tiles* t, const double* d_x, const double* d_y, geo_theta theta, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_x) return -2;
    if (!d_y) return -3;
    if (check_theta(theta)) return -4;
    Layout L = make_layout(t);
    return launch_matern_tiles(L, d_x, d_y, theta, nullptr, 0, (cudaStream_t)stream) ? GEO_ERR_CUDA : GEO_OK;
}

int geo_tiles_load_dense(geo_tiles* t, const double* d_a, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_a) return -2;
    return launch_load_dense(make_layout(t), d_a, (cudaStream_t)stream) ? GEO_ERR_CUDA : GEO_OK;
}

int geo_tiles_to_dense(const geo_tiles* t, double* d_out, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_out) return -2;
    return launch_to_dense(make_layout(t), d_out, (cudaStream_t)stream) ? GEO_ERR_CUDA : GEO_OK;
}

// status words and the per-step work tickets of the persistent update kernels
static int reset_status(const Layout& L, cudaStream_t s) {
    return cudaMemsetAsync(L.status, 0, sizeof(int) * ((size_t)ST_WORDS + 2 * (size_t)L.p), s) ? GEO_ERR_CUDA
                                                                                                 : GEO_OK;
}

// Algorithm 1 on the store.  With z, the persistent tile-DAG path also runs the
// forward solve of Eq. 2 inside the same launch and writes (log|Sigma|,
// Z' Sigma^-1 Z) to res; *solved tells the caller whether that happened (the
// step-by-step paths leave the solve to run_logdet_trsv).
// scheduling variant of a bound store: in-band updates on the tensor cores (0)
// unless the FP64 pipe is asked for or there are no slice planes (a single
// tile: 1); the DST approximation (2)
static int sched_variant(const geo_tiles* t) {
    if (!t->d_planes || t->lay.bytes_planes == 0) return 1;
    if (t->flags & GEO_FLAG_DST) return 2;
    return (t->flags & GEO_FLAG_FP64_DMMA) ? 1 : 0;
}

static cudaError_t factor(const geo_tiles* t, const Layout& L, const double* z, double* res, bool* solved,
                          cudaStream_t s) {
    *solved = false;
    if (L.lp_mode == GEO_LP_SPLIT_BF16 && !(t->flags & GEO_FLAG_STEPWISE)) {
        MetaOffsets mo = meta_offsets(t->lay);
        const int v = sched_variant(t);
        SchedView sv;
        sv.geom = mo.geom[v];
        char* base = (char*)t->d_meta;
        sv.counters = (int*)(base + mo.sched_ctr);
        sv.prio = (const G2Task*)(base + mo.sched_g2[v]);
        sv.bulk = (const G2Task*)(base + mo.sched_bulk[v]);
        sv.trsm_end = (const int*)(base + mo.sched_end[v]);
        sv.tct = (const int4*)(base + mo.sched_tct[v]);
        sv.yq = (const G2Task*)(base + mo.sched_y[v]);
        *solved = z != nullptr;
        return run_potrf_dag(t, L, sv, z, res, s);
    }
    return run_potrf_mp(t, L, s);
}

int geo_potrf_mp(geo_tiles* t, void* stream) {
    if (check_bound(t)) return -1;
    Layout L = make_layout(t);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = reset_status(L, s);
    if (rc) return rc;
    bool solved = false;
    return factor(t, L, nullptr, nullptr, &solved, s) ? GEO_ERR_CUDA : GEO_OK;
}

int geo_logdet_trsv(const geo_tiles* t, const double* d_z, double* d_logdet, double* d_quad, double* d_y,
                    void* stream) {
    if (check_bound(t)) return -1;
    if (!d_z) return -2;
    if (!d_logdet) return -3;
    if (!d_quad) return -4;
    return run_logdet_trsv(make_layout(t), d_z, d_logdet, d_quad, d_y, (cudaStream_t)stream) ? GEO_ERR_CUDA
                                                                                             : GEO_OK;
}

int geo_logdet_trsv_noalloc(const geo_tiles* t, const double* d_z, double* d_logdet, double* d_quad,
                            void* stream) {
    if (check_bound(t)) return -1;
    if (!d_z) return -2;
    if (!d_logdet) return -3;
    if (!d_quad) return -4;
    const long long np = (long long)t->lay.p * t->lay.nb;
    if (np > GEO_NOALLOC_MAX_N || t->lay.p > GEO_NOALLOC_MAX_P) return GEO_ERR_TOO_LARGE;
    return run_logdet_trsv_noalloc(make_layout(t), d_z, d_logdet, d_quad, (cudaStream_t)stream) ? GEO_ERR_CUDA
                                                                                                : GEO_OK;
}

int geo_status(const geo_tiles* t, int* h_code, int* h_info, void* stream) {
    if (check_bound(t)) return -1;
    if (!h_code) return -2;
    Layout L = make_layout(t);
    int st[3] = {0, 0, 0};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(st, L.status, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return GEO_ERR_CUDA;
    *h_code = st[ST_CODE];
    if (h_info) *h_info = st[ST_CODE] == GEO_ERR_TIMEOUT ? st[ST_TIMEOUT_WHERE] : st[ST_INFO];
    return GEO_OK;
}

// d_res[0..2] = (log|Sigma|, Z' Sigma^-1 Z, Eq. 2), all three NaN when the
// factorization fails: they start as NaN (every byte 0xFF) and only the
// solve's last step, which runs after every tile was factored, writes them.
static int loglik_enqueue(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta,
                          double* d_res, cudaStream_t s) {
    Layout L = make_layout(t);
    int rc = reset_status(L, s);
    if (rc) return rc;
    if (cudaMemsetAsync(d_res, 0xFF, 3 * sizeof(double), s)) return GEO_ERR_CUDA;
    prof_begin(5, s);
    const cudaError_t eg = launch_matern_tiles(L, d_x, d_y, theta, nullptr, 0, s);
    prof_end(5, s);
    if (eg) return GEO_ERR_CUDA;
    bool solved = false;
    if (factor(t, L, d_z, d_res, &solved, s)) return GEO_ERR_CUDA;
    if (!solved && run_logdet_trsv(L, d_z, d_res, d_res + 1, nullptr, s, d_res + 2)) return GEO_ERR_CUDA;
    return GEO_OK;
}

int geo_loglik_async(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta,
                     double* d_res, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_x) return -2;
    if (!d_y) return -3;
    if (!d_z) return -4;
    if (check_theta(theta)) return -5;
    if (!d_res) return -6;
    return loglik_enqueue(t, d_x, d_y, d_z, theta, d_res, (cudaStream_t)stream);
}

int geo_loglik(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta,
               double* h_out, int* h_info, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_x) return -2;
    if (!d_y) return -3;
    if (!d_z) return -4;
    if (check_theta(theta)) return -5;
    if (!h_out) return -6;
    Layout L = make_layout(t);
    cudaStream_t s = (cudaStream_t)stream;
    double* res = L.scal + 2 * L.p;
    const int rc = loglik_enqueue(t, d_x, d_y, d_z, theta, res, s);
    if (rc) return rc;
    double hres[3];
    int st[2];
    cudaError_t e = cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(st, L.status, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return GEO_ERR_CUDA;
    if (h_info) *h_info = st[1];
    if (st[0] != 0) return st[0];
    h_out[0] = hres[2];   // Eq. 2, assembled on the device
    h_out[1] = hres[0];
    h_out[2] = hres[1];
    return GEO_OK;
}

int geo_krige(const geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta,
              const double* d_xnew, const double* d_ynew, int m, double* d_zhat, double* d_work, void* stream) {
    if (check_bound(t)) return -1;
    if (!d_x) return -2;
    if (!d_y) return -3;
    if (!d_z) return -4;
    if (check_theta(theta)) return -5;
    if (m < 0) return -8;
    if (m > 0 && (!d_xnew || !d_ynew)) return -6;
    if (m > 0 && !d_zhat) return -9;
    if (!d_work) return -10;
    return run_krige(make_layout(t), d_x, d_y, d_z, make_matern(theta), d_xnew, d_ynew, m, d_zhat, d_work,
                     (cudaStream_t)stream)
               ? GEO_ERR_CUDA
               : GEO_OK;
}

unsigned long long geo_kernel_launches(void) { return g_launches.load(); }

int geo_profile_enable(int on) {
    g_prof = on != 0;
    return GEO_OK;
}

int geo_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& sl : g_slots) {
        prof_collect(sl);
        sl.ms = 0.0;
        sl.launches = 0;
    }
    return GEO_OK;
}

int geo_profile_read(int kind, double* h_ms, long long* h_launches) {
    if (kind < 0 || kind > 5) return -1;
    if (!h_ms) return -2;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_collect(g_slots[kind]);
    *h_ms = g_slots[kind].ms;
    if (h_launches) *h_launches = g_slots[kind].launches;
    return GEO_OK;
}

}  // extern "C"

// ---- batched evaluation ------------------------------------------------------
namespace {
struct BatchMeta {
    int nprob;
    size_t off_probs, off_maps, off_tend, off_prio, off_bulk, off_tct, off_y, off_gen, off_ctr, total;
    long long n_prio, n_bulk, n_tct, n_y;
    long long gen_blocks;   // CTAs of the batch's one generator launch
    int per;
    size_t counter_bytes;
    int ctas;   // CTAs of the factorization launch (0: one per SM, cooperative)
};
std::mutex g_batch_mu;
std::vector<std::pair<const void*, BatchMeta>> g_batches;   // bound workspaces

int batch_variant(const geo_tiles* t) { return sched_variant(t); }

int batch_meta(int nprob, const geo_batch_item* items, BatchMeta& m, std::vector<SchedGeom>* geoms) {
    if (nprob < 1) return -1;
    if (!items) return -2;
    m = BatchMeta();
    m.nprob = nprob;
    long long ptot = 0, ctot = 16;
    m.n_prio = m.n_bulk = m.n_tct = m.n_y = 0;
    m.per = 1;
    for (int b = 0; b < nprob; ++b) {
        const geo_batch_item& it = items[b];
        if (!it.t || !it.t->d_meta || !it.d_x || !it.d_y || !it.d_z) return -2;
        if (it.t->lay.lp_mode != GEO_LP_SPLIT_BF16) return -2;   // the batch runs the tensor-core DAG path
        const MetaOffsets mo = meta_offsets(it.t->lay);
        const SchedGeom& g = mo.geom[batch_variant(it.t)];
        if (geoms) geoms->push_back(g);
        ptot += g.p;
        ctot += g.n_counters - 16;
        m.n_prio += g.n_prio;
        m.n_bulk += g.n_bulk;
        m.n_tct += g.n_tct;
        m.n_y += g.n_y;
        m.per = std::max(m.per, g.items_tc);
    }
    size_t b = 0;
    m.off_probs = b;
    b = align256(b + sizeof(ProbDev) * (size_t)nprob);
    m.off_maps = b;
    b = align256(b + sizeof(CUtensorMap) * 3 * (size_t)nprob);
    m.off_tend = b;
    b = align256(b + sizeof(int) * (size_t)ptot);
    m.off_prio = b;
    b = align256(b + sizeof(G2Task) * (size_t)std::max(m.n_prio, 1LL));
    m.off_bulk = b;
    b = align256(b + sizeof(G2Task) * (size_t)std::max(m.n_bulk, 1LL));
    m.off_tct = b;
    b = align256(b + sizeof(int4) * (size_t)std::max(m.n_tct, 1LL));
    m.off_y = b;
    b = align256(b + sizeof(G2Task) * (size_t)std::max(m.n_y, 1LL));
    m.off_gen = b;
    b = align256(b + sizeof(GenJob) * (size_t)nprob);
    m.off_ctr = b;
    m.counter_bytes = sizeof(int) * (size_t)ctot;
    b = align256(b + m.counter_bytes);
    m.total = b;
    return 0;
}
}  // namespace

extern "C" {

int geo_batch_workspace(int nprob, const geo_batch_item* items, size_t* bytes) {
    if (!bytes) return -3;
    BatchMeta m;
    const int rc = batch_meta(nprob, items, m, nullptr);
    if (rc) return rc;
    *bytes = m.total;
    return GEO_OK;
}

int geo_batch_bind(int nprob, const geo_batch_item* items, void* d_work, size_t bytes, void* stream) {
    BatchMeta m;
    std::vector<SchedGeom> geoms;
    int rc = batch_meta(nprob, items, m, &geoms);
    if (rc) return rc;
    if (!d_work) return -3;
    if (bytes < m.total) return -4;
    std::vector<int> bands((size_t)nprob);
    for (int b = 0; b < nprob; ++b) bands[(size_t)b] = items[b].t->lay.band;
    BatchPlan plan;
    sched_merge(geoms, bands, plan);
    if ((long long)plan.prio.size() != m.n_prio || (long long)plan.bulk.size() != m.n_bulk ||
        (long long)plan.tct.size() != m.n_tct || (long long)plan.yq.size() != m.n_y || plan.per != m.per)
        return GEO_ERR_UNSUPPORTED;   // the merge must account for every task
    char* base = (char*)d_work;
    std::vector<ProbDev> probs((size_t)nprob);
    std::vector<CUtensorMap> maps(3 * (size_t)nprob);
    std::vector<GenJob> gen((size_t)nprob);
    std::vector<int> tend;
    long long gblk = 0;
    int* ctr = (int*)(base + m.off_ctr) + 16;
    for (int b = 0; b < nprob; ++b) {
        const geo_tiles* t = items[b].t;
        ProbDev& P = probs[(size_t)b];
        memset(&P, 0, sizeof(P));
        P.L = make_layout(t);
        P.g = geoms[(size_t)b];
        bind_counters(P, ctr);
        ctr += P.g.n_counters - 16;
        P.trsm_end = (const int*)(base + m.off_tend) + tend.size();
        tend.insert(tend.end(), plan.trsm_end[(size_t)b].begin(), plan.trsm_end[(size_t)b].end());
        P.tmap = (const CUtensorMap*)(base + m.off_maps) + 3 * (size_t)b;
        memcpy(&maps[3 * (size_t)b], t->tmap, 3 * sizeof(CUtensorMap));
        P.z = items[b].d_z;   // the forward solve runs inside the launch
        P.y0 = plan.ybeg[(size_t)b];
        P.y1 = plan.ybeg[(size_t)b + 1];
        gen[(size_t)b] = {items[b].d_x, items[b].d_y, gblk};
        gblk += gen_blocks(P.L);
    }
    if (gblk > 0x7fffffffLL) return GEO_ERR_TOO_LARGE;   // one generator launch holds every problem's CTAs
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(base + m.off_probs, probs.data(), sizeof(ProbDev) * probs.size(),
                                    cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + m.off_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                cudaMemcpyHostToDevice, s);
    if (!e && !tend.empty())
        e = cudaMemcpyAsync(base + m.off_tend, tend.data(), sizeof(int) * tend.size(), cudaMemcpyHostToDevice, s);
    if (!e && !plan.prio.empty())
        e = cudaMemcpyAsync(base + m.off_prio, plan.prio.data(), sizeof(G2Task) * plan.prio.size(),
                            cudaMemcpyHostToDevice, s);
    if (!e && !plan.bulk.empty())
        e = cudaMemcpyAsync(base + m.off_bulk, plan.bulk.data(), sizeof(G2Task) * plan.bulk.size(),
                            cudaMemcpyHostToDevice, s);
    if (!e && !plan.tct.empty())
        e = cudaMemcpyAsync(base + m.off_tct, plan.tct.data(), sizeof(int4) * plan.tct.size(),
                            cudaMemcpyHostToDevice, s);
    if (!e && !plan.yq.empty())
        e = cudaMemcpyAsync(base + m.off_y, plan.yq.data(), sizeof(G2Task) * plan.yq.size(),
                            cudaMemcpyHostToDevice, s);
    if (!e)
        e = cudaMemcpyAsync(base + m.off_gen, gen.data(), sizeof(GenJob) * gen.size(), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return GEO_ERR_CUDA;
    m.ctas = 0;
    m.gen_blocks = gblk;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& kv : g_batches)
        if (kv.first == d_work) {
            kv.second = m;
            return GEO_OK;
        }
    g_batches.push_back({d_work, m});
    return GEO_OK;
}

int geo_batch_set_ctas(const void* d_work, int ctas) {
    if (!d_work) return -1;
    if (ctas < 0 || (ctas > 0 && ctas < GEO_MIN_CTAS)) return -2;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& kv : g_batches)
        if (kv.first == d_work) {
            kv.second.ctas = ctas;
            return GEO_OK;
        }
    return -1;   // not bound by geo_batch_bind
}

int geo_batch_release(const void* d_work) {
    if (!d_work) return -1;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t q = 0; q < g_batches.size(); ++q)
        if (g_batches[q].first == d_work) {
            g_batches.erase(g_batches.begin() + (long)q);
            return GEO_OK;
        }
    return -1;
}

int geo_loglik_batch(int nprob, const geo_batch_item* items, const geo_theta* d_theta, void* d_work,
                     double* d_out, long long* d_done_ns, void* stream) {
    if (nprob < 1) return -1;
    if (!items) return -2;
    if (!d_theta) return -3;
    if (!d_work) return -4;
    if (!d_out) return -5;
    BatchMeta m;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        bool found = false;
        for (auto& kv : g_batches)
            if (kv.first == d_work) {
                m = kv.second;
                found = true;
            }
        if (!found || m.nprob != nprob) return -4;   // not bound by geo_batch_bind for this batch
    }
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)d_work;
    bool small_dp = false;
    for (int b = 0; b < nprob; ++b) {
        const Layout L = make_layout(items[b].t);
        small_dp = small_dp || dag_small_dp(L.nb, L.band);
    }
    // every problem's generation in one launch (theta from d_theta[b])
    if (launch_matern_batch((const ProbDev*)(base + m.off_probs), (const GenJob*)(base + m.off_gen), nprob,
                            m.gen_blocks, d_theta, s))
        return GEO_ERR_CUDA;
    if (run_potrf_dag_batch((const ProbDev*)(base + m.off_probs), nprob, (const G2Task*)(base + m.off_prio),
                            m.n_prio, (const G2Task*)(base + m.off_bulk), m.n_bulk,
                            (const int4*)(base + m.off_tct), m.n_tct, m.per, (const G2Task*)(base + m.off_y),
                            m.n_y, d_out, d_done_ns, (int*)(base + m.off_ctr), m.counter_bytes,
                            items[0].t->trace, items[0].t->trace_cap, small_dp, items[0].t->timeout_ns, m.ctas, s))
        return GEO_ERR_CUDA;
    return GEO_OK;
}

}  // extern "C"
