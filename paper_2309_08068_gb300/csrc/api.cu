// C-ABI of liblbm.so (declared in include/lbm.h): context lifecycle, argument checks, media
// compression, source bookkeeping and kernel dispatch. No call aborts; every failure returns an
// LBM_E* code with a message kept on the context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

using namespace lbm;

namespace {

struct HostSource {
    int kind;
    std::vector<int> cells;
    std::vector<float> w;  // 3 per cell (current)
    float E0[3], B0[3];
    lbm_time_fn fn;
    std::vector<double> table;
};

thread_local std::string g_create_error;

}  // namespace

struct lbm_ctx {
    int model = 0;
    Geometry g{};
    cudaStream_t stream = nullptr;
    int track_rho = 0;
    int z_ghost = 0;  // z-slab with ghost planes 0 and nz - 1 (stepped planes 1 .. nz - 2)
    double eps0 = 0, mu0 = 0;
    int device = 0;
    int storage = LBM_F32;
    float scale = 1.f;
    // populations (pull scheme, two buffers)
    void* buf[2] = {nullptr, nullptr};   // MM float4[12][n]; HV float4[6][n]
    void* buf2[2] = {nullptr, nullptr};  // HV float2[6][n]
    float* rho[2] = {nullptr, nullptr};  // MM f_0^(0) (track_rho)
    float* rest1 = nullptr;              // MM f_0^(1) (track_rho)
    int cur = 0;
    // media
    int media_mode = kUniform;
    MatCoef uniform{};
    uint8_t* mat_id = nullptr;
    MatCoef* mat_table = nullptr;
    float* eps_r = nullptr;
    float* mu_r = nullptr;
    float* sigma = nullptr;
    // sources
    std::vector<HostSource> sources;
    int n_special = 0;
    int* d_cell = nullptr;
    int* d_entry_begin = nullptr;
    int* d_entry_src = nullptr;
    float* d_entry_w = nullptr;
    uint32_t* d_impose_mask = nullptr;
    int* d_block_begin = nullptr;  // where each kBlock-cell block of the step range starts in d_cell
    // reductions
    double* d_partials = nullptr;
    double* d_result = nullptr;
    int reduce_blocks = 0;
    int partial_capacity = 0;  // blocks
    // adjoint work space (records, checkpoints, adjoint states), kept between lbm_adjoint calls
    void* adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
    float* host_stage = nullptr;  // device staging of host fields for lbm_init_fields / lbm_fields
    size_t host_stage_bytes = 0;
    // staging of a packed halo face for host-side lbm_halo_pack / lbm_halo_unpack
    void* halo_stage = nullptr;
    size_t halo_stage_bytes = 0;
    // two steps per pass (lbm_step with n >= 2): mode, intermediate planes, counters
    int fusion = 1;                // 0 off, 1 automatic, 2 the L2-ring pass, 3 the tiled pass, when possible
    int fused_tile = 0;            // cells per work item of a pass (0: the model's default)
    void* fused_planes = nullptr;  // R ring slots + the slots of planes 0 and nz - 1
    size_t fused_planes_bytes = 0;
    int* fused_ctrl = nullptr;     // item counter, abort, 2 nz tiles tile flags
    int fused_epoch = 0;           // number of the last pass launched
    int* d_tile_special = nullptr;  // nz tiles + 1 offsets of each tile's cells in the special-cell list
    int* d_tiled_off = nullptr;     // tiled pass: tiles nz + 1 offsets into d_tiled_entries, by (tile, plane)
    int2* d_tiled_entries = nullptr;  // tiled pass: (special-cell index, extended-tile position)
    int tiled_version = -1;           // sources_version the two arrays were built for
    int tile_special_version = -1;   // sources_version it was built for (-1: rebuild)
    int sources_version = 0;
    int fused_pending = 0;         // a pass ran since the abort flag was last read
    long long wait_limit_ns = 0;   // dependency-wait limit of a pass (0: the default)
    std::vector<int> h_cell;       // host copy of the special-cell list (sorted)
    int64_t t = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

int fail(lbm_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_error = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                         \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail((ctx), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int check_launch(lbm_ctx* ctx, int launched) {
    ctx->launches += launched;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, LBM_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}


int ensure_device(lbm_ctx* ctx) {
    int dev = -1;
    CUDA_TRY(ctx, cudaGetDevice(&dev));
    if (dev != ctx->device) CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return LBM_OK;
}

// Bytes per cell of the main population array (MM: 12 groups of 4; HV: 6 groups of 4) and of HV's
// second array (6 groups of 2).
// LBM_F24 keeps 3 bytes per value: a plane of halves and a plane of correction bytes per group.
size_t group_bytes(int model, int storage) {
    const size_t v4 = storage == LBM_F32 ? sizeof(float4) : (storage == LBM_F24 ? 4 * 3 : 4 * sizeof(uint16_t));
    return model == LBM_MM ? 12 * v4 : 6 * v4;
}
size_t pair_bytes(int storage) {
    return 6 * (storage == LBM_F32 ? sizeof(float2) : (storage == LBM_F24 ? 2 * 3 : 2 * sizeof(uint16_t)));
}

StepArgs base_args(lbm_ctx* c) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.g = c->g;
    a.cell_begin = c->z_ghost ? c->g.nx * c->g.ny : 0;
    a.cell_end = c->z_ghost ? c->g.n - c->g.nx * c->g.ny : c->g.n;
    a.media_mode = c->media_mode;
    a.media.uniform = c->uniform;
    a.media.id = c->mat_id;
    a.media.table = c->mat_table;
    a.media.eps_r = c->eps_r;
    a.media.mu_r = c->mu_r;
    a.media.sigma = c->sigma;
    a.sv.n_special = c->n_special;
    a.sv.cell = c->d_cell;
    a.sv.entry_begin = c->d_entry_begin;
    a.sv.entry_src = c->d_entry_src;
    a.sv.entry_w = c->d_entry_w;
    a.sv.impose_mask = c->d_impose_mask;
    a.sv.block_begin = c->d_block_begin;
    for (size_t k = 0; k < c->sources.size(); ++k) {
        for (int q = 0; q < 3; ++q) {
            a.sc.E0[k][q] = c->sources[k].E0[q];
            a.sc.B0[k][q] = c->sources[k].B0[q];
        }
    }
    a.eps0 = (float)c->eps0;
    a.mu0 = (float)c->mu0;
    a.storage = c->storage;
    a.scale = c->scale;
    a.inv_scale = 1.f / c->scale;
    return a;
}

// Current buffer as input (fin*) and the other as output (fout*).
void bind_buffers(lbm_ctx* c, StepArgs& a, int in, int out) {
    a.fin = c->buf[in];
    a.fout = c->buf[out];
    if (c->model == LBM_HV) {
        a.fin2 = c->buf2[in];
        a.fout2 = c->buf2[out];
    } else {
        a.fin2 = c->rest1;
        a.fout2 = c->rest1;
    }
    a.rho_in = c->rho[in];
    a.rho_out = c->rho[out];
}

double time_value(const HostSource& s, int64_t t) {
    const double pi = 3.14159265358979323846;
    switch (s.fn.kind) {
        case LBM_FN_SIN: return s.fn.amplitude * std::sin(2.0 * pi * (double)t / s.fn.period + s.fn.phase);
        case LBM_FN_TABLE:
            return (t >= 0 && t < (int64_t)s.table.size()) ? s.fn.amplitude * s.table[(size_t)t] : 0.0;
        default: return s.fn.amplitude;
    }
}

void fill_scalars(lbm_ctx* c, StepArgs& a, int64_t t) {
    for (size_t k = 0; k < c->sources.size(); ++k) a.sc.s[k] = (float)time_value(c->sources[k], t);
}

template <class T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// --- two steps per pass ------------------------------------------------------------------------
// Pass shape per model, measured on GB300 (256^3 dipole): the ring slots R (planes 1 .. nz - 2),
// the lookahead L of A phases over B phases (R >= L + 1), and the cells per work item. Deeper
// rings let more work run at once until the ring no longer stays in L2.
struct FusedShape {
    int R, L, tile;
};
constexpr FusedShape kFusedMM{5, 3, 256};
constexpr FusedShape kFusedHV{6, 4, 512};
static_assert(kFusedMM.L >= 2 && kFusedMM.R >= kFusedMM.L + 1 && kFusedHV.L >= 2 && kFusedHV.R >= kFusedHV.L + 1,
              "the pass order needs R >= L + 1 >= 3");
constexpr long long kFusedTimeoutNs = 2000000000;  // a dependency wait longer than this aborts

FusedShape fused_shape(const lbm_ctx* c) { return c->model == LBM_MM ? kFusedMM : kFusedHV; }

int fused_tile_cells(const lbm_ctx* c) { return c->fused_tile ? c->fused_tile : fused_shape(c).tile; }
int fused_tiles(const lbm_ctx* c) { return (c->g.nx * c->g.ny + fused_tile_cells(c) - 1) / fused_tile_cells(c); }

// Pass control block: [item counter][abort][2 nz x tiles tile flags]. The item counter is zeroed
// before every pass; the abort flag stays set until check_fused_abort reports it.
size_t fused_ctrl_ints(const lbm_ctx* c) {
    const size_t nz = (size_t)c->g.nz, tiles = (size_t)fused_tiles(c);
    return 2 + 2 * nz * tiles;
}

size_t fused_plane_bytes(const lbm_ctx* c) {
    const size_t nxy = (size_t)c->g.nx * c->g.ny;
    return (group_bytes(c->model, c->storage) + (c->model == LBM_HV ? pair_bytes(c->storage) : 0)) * nxy;
}

// The L2-ring pass applies when the wavefront has enough tiles per plane to fill the GPU and, by
// default, the populations are stored in FP32 and the intermediate planes fit in three quarters of
// L2, where they are meant to stay.
bool ring_eligible(const lbm_ctx* c) {
    if (c->fusion == 0 || c->fusion == 3 || c->z_ghost || c->track_rho || c->storage == LBM_F24 ||
        c->g.nz < std::max(3, fused_shape(c).L + 1))
        return false;
    int dev = 0, sms = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (c->g.nx * c->g.ny < sms * kBlock) return false;
    if (c->fusion == 1 && (fused_shape(c).R + 2) * fused_plane_bytes(c) > (size_t)l2 / 4 * 3) return false;
    // With 16-bit storage the single-step kernels move so few bytes that they beat the pass, whose
    // time is set by its wavefront's latency, not by its bytes (256^3 dipole on GB300: MM 0.50 ms
    // per step against 0.62, HV 0.36 against 0.49).
    if (c->fusion == 1 && c->storage != LBM_F32) return false;
    return true;
}

// The tiled pass needs a whole extended tile of distinct cells in x and y.
bool tiled_possible(const lbm_ctx* c) {
    return !c->z_ghost && !c->track_rho && c->storage != LBM_F24 && c->g.nz >= 3 && c->g.nx >= kTileEX &&
           c->g.ny >= kTileEY;
}

// Whether a tiled pass has more than 1.5 waves of resident blocks at its shortest chunks (8 planes).
// Below that its extra phase-A planes and a ragged last wave cost more than the second step saves:
// on GB300 it measured slower than single steps on 32^3 to 80^3 lattices (MM 32^3: 13.3 us per step
// against 6.2) and on 256 x 160 x 16 (MM 49.1 us against 42.7), faster from 96^3 (MM, 1.9 waves).
bool tiled_fills(const lbm_ctx* c) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int occ = std::max(1, c->model == LBM_MM ? mm_tile2_occupancy(c->storage, c->media_mode)
                                                   : hv_tile2_occupancy(c->storage, c->media_mode));
    const long long tiles = (long long)((c->g.nx + kTileTX - 1) / kTileTX) * ((c->g.ny + kTileTY - 1) / kTileTY);
    const long long blocks = tiles * ((c->g.nz + 7) / 8);
    return 2 * blocks > 3LL * sms * occ;
}

enum { kPassNone = 0, kPassRing = 1, kPassTiled = 2 };

// Which two-step pass lbm_step(n >= 2) runs: mode 2 the ring, mode 3 the tiles, wherever each is
// possible. Mode 1 takes what measured fastest on GB300 with FP32 storage (ms per step):
//   MM: the tiled pass where it fills the GPU (256^3 dipole: 0.607 against 0.763 for the ring pass
//   and 0.925 for single steps; 128^3: 0.093 against 0.103), else the ring pass where it applies.
//   HV, uniform medium: the ring pass where it applies (256^3 dipole: 0.517 against 0.540 for the
//   tiled pass, which is held by shared-memory instruction throughput), else the tiled pass where
//   it fills the GPU (128^3: 0.085 against 0.090 for single steps).
//   HV, other media: the tiled pass first (272^3 skin-effect lattice with a material table: 0.630
//   against 0.696 for the ring pass; 208^3: 0.317 against 0.343), then the ring pass.
// Where none applies, single steps.
int pass_kind(const lbm_ctx* c) {
    if (c->fusion == 0) return kPassNone;
    if (c->fusion == 3) return tiled_possible(c) ? kPassTiled : kPassNone;
    if (c->fusion == 2) return ring_eligible(c) ? kPassRing : kPassNone;
    if (c->storage != LBM_F32) return kPassNone;  // 16-bit storage: single steps (see ring_eligible)
    const bool ring_first = c->model == LBM_HV && c->media_mode == kUniform;
    if (ring_first && ring_eligible(c)) return kPassRing;
    if (tiled_possible(c) && tiled_fills(c)) return kPassTiled;
    return ring_eligible(c) ? kPassRing : kPassNone;
}

int ensure_fused(lbm_ctx* c) {
    const size_t need = (fused_shape(c).R + 2) * fused_plane_bytes(c);
    if (c->fused_planes_bytes < need) {
        free_dev(c->fused_planes);
        c->fused_planes_bytes = 0;
        if (cudaMalloc(&c->fused_planes, need) != cudaSuccess) {
            cudaGetLastError();
            c->fused_planes = nullptr;
            return fail(c, LBM_ENOMEM, "lbm_step: cannot allocate %zu bytes of intermediate planes", need);
        }
        c->fused_planes_bytes = need;
    }
    if (!c->fused_ctrl) {
        const size_t ints = fused_ctrl_ints(c);
        if (cudaMalloc(&c->fused_ctrl, sizeof(int) * ints) != cudaSuccess) {
            cudaGetLastError();
            c->fused_ctrl = nullptr;
            return fail(c, LBM_ENOMEM, "lbm_step: cannot allocate the pass counters");
        }
        CUDA_TRY(c, cudaMemsetAsync(c->fused_ctrl, 0, sizeof(int) * ints, c->stream));
        c->fused_epoch = 0;
    }
    if (c->tile_special_version != c->sources_version || !c->d_tile_special) {
        // offsets of each tile's cells in the sorted special-cell list: tile j of plane p holds cells
        // p nxy + j tile_cells .. (up to the end of the plane)
        const int nz = c->g.nz, nxy = c->g.nx * c->g.ny, tiles = fused_tiles(c), tc = fused_tile_cells(c);
        std::vector<int> off((size_t)nz * tiles + 1, 0);
        size_t m = 0;
        for (size_t k = 0; k <= (size_t)nz * tiles; ++k) {
            const int p = (int)(k / tiles), j = (int)(k % tiles);
            const long long start = (long long)p * nxy + std::min((long long)j * tc, (long long)nxy);
            while (m < c->h_cell.size() && c->h_cell[m] < start) ++m;
            off[k] = (int)m;
        }
        free_dev(c->d_tile_special);
    free_dev(c->d_tiled_off);
    free_dev(c->d_tiled_entries);
        if (cudaMalloc(&c->d_tile_special, sizeof(int) * off.size()) != cudaSuccess) {
            cudaGetLastError();
            c->d_tile_special = nullptr;
            return fail(c, LBM_ENOMEM, "lbm_step: cannot allocate the tiles' source-cell offsets");
        }
        CUDA_TRY(c, cudaMemcpy(c->d_tile_special, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
        c->tile_special_version = c->sources_version;
    }
    return LBM_OK;
}

int fused_pass(lbm_ctx* c) {
    const int in = c->cur, out = 1 - c->cur;
    StepArgs aA = base_args(c), aB = base_args(c);
    bind_buffers(c, aA, in, out);
    bind_buffers(c, aB, in, out);
    fill_scalars(c, aA, c->t + 1);
    fill_scalars(c, aB, c->t + 2);
    const size_t nxy = (size_t)c->g.nx * c->g.ny;
    const size_t g_plane = group_bytes(c->model, c->storage) * nxy;
    const size_t p_plane = c->model == LBM_HV ? pair_bytes(c->storage) * nxy : 0;
    const FusedShape shape = fused_shape(c);
    const int R = shape.R;
    char* base = static_cast<char*>(c->fused_planes);
    char* groups = base;                        // R + 2 group planes
    char* pairs = base + (R + 2) * g_plane;     // R + 2 pair planes (HV)
    FusedArgs F;
    memset(&F, 0, sizeof(F));
    F.ring = groups;
    F.lo = groups + R * g_plane;
    F.hi = groups + (R + 1) * g_plane;
    if (p_plane) {
        F.ring2 = pairs;
        F.lo2 = pairs + R * p_plane;
        F.hi2 = pairs + (R + 1) * p_plane;
    }
    F.R = R;
    F.L = shape.L;
    F.tile_cells = fused_tile_cells(c);
    F.tiles = fused_tiles(c);
    F.epoch = ++c->fused_epoch;
    F.next = c->fused_ctrl;
    F.abort = c->fused_ctrl + 1;
    F.tile_flag = c->fused_ctrl + 2;
    F.tile_special = c->d_tile_special;
    F.timeout_ns = c->wait_limit_ns ? c->wait_limit_ns : kFusedTimeoutNs;
    CUDA_TRY(c, cudaMemsetAsync(c->fused_ctrl, 0, sizeof(int), c->stream));
    const int launched = c->model == LBM_MM ? mm_launch_fused2(aA, aB, F, c->stream) : hv_launch_fused2(aA, aB, F, c->stream);
    int rc = check_launch(c, launched);
    if (rc != LBM_OK) return rc;
    c->fused_pending = 1;
    c->cur = out;
    c->t += 2;
    return LBM_OK;
}

// Reports (once) a two-step pass whose dependency wait timed out since the last check.
int check_fused_abort(lbm_ctx* c) {
    if (!c->fused_pending || !c->fused_ctrl) return LBM_OK;
    int flag = 0;
    int* abort = c->fused_ctrl + 1;
    CUDA_TRY(c, cudaMemcpyAsync(&flag, abort, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->fused_pending = 0;
    if (flag) {
        CUDA_TRY(c, cudaMemsetAsync(abort, 0, sizeof(int), c->stream));
        return fail(c, LBM_ETIMEDOUT,
                    "a two-step pass stopped: a dependency wait exceeded its time limit; the populations "
                    "of that pass are undefined (restore them with lbm_set_populations)");
    }
    return LBM_OK;
}

// --- two steps per pass over shared-memory tiles ----------------------------------------------
int tiled_tiles_x(const lbm_ctx* c) { return (c->g.nx + kTileTX - 1) / kTileTX; }
int tiled_tiles_y(const lbm_ctx* c) { return (c->g.ny + kTileTY - 1) / kTileTY; }

// The source cells of every tile's extended cells, by (tile, plane): the tiled pass recomputes them
// after each ordinary update of their plane.
int ensure_tiled(lbm_ctx* c) {
    if (c->tiled_version == c->sources_version && c->d_tiled_off) return LBM_OK;
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz, nxy = nx * ny;
    const int tx = tiled_tiles_x(c), ty = tiled_tiles_y(c);
    // extended positions (tile, position) at which each lattice x, and each y, appears
    std::vector<std::vector<std::pair<int, int>>> xs((size_t)nx), ys((size_t)ny);
    for (int b = 0; b < tx; ++b)
        for (int e = 0; e < kTileEX; ++e) xs[(size_t)tile_coord(b, e, kTileTX, nx)].emplace_back(b, e);
    for (int b = 0; b < ty; ++b)
        for (int e = 0; e < kTileEY; ++e) ys[(size_t)tile_coord(b, e, kTileTY, ny)].emplace_back(b, e);
    struct Entry {
        long long key;  // tile nz + plane
        int m, local;
    };
    std::vector<Entry> entries;
    for (size_t m = 0; m < c->h_cell.size(); ++m) {
        const int cell = c->h_cell[m], z = cell / nxy, r = cell - z * nxy, y = r / nx, x = r - y * nx;
        for (const auto& px : xs[(size_t)x])
            for (const auto& py : ys[(size_t)y])
                entries.push_back(Entry{(long long)(px.first + tx * py.first) * nz + z, (int)m,
                                        px.second + kTileEX * py.second});
    }
    std::stable_sort(entries.begin(), entries.end(), [](const Entry& a, const Entry& b) { return a.key < b.key; });
    const size_t keys = (size_t)tx * ty * nz;
    std::vector<int> off(keys + 1, 0);
    std::vector<int2> list(std::max<size_t>(entries.size(), 1));
    for (size_t k = 0; k < entries.size(); ++k) {
        off[(size_t)entries[k].key + 1] += 1;
        list[k] = make_int2(entries[k].m, entries[k].local);
    }
    for (size_t k = 0; k < keys; ++k) off[k + 1] += off[k];
    free_dev(c->d_tiled_off);
    free_dev(c->d_tiled_entries);
    if (cudaMalloc(&c->d_tiled_off, sizeof(int) * off.size()) != cudaSuccess ||
        cudaMalloc(&c->d_tiled_entries, sizeof(int2) * list.size()) != cudaSuccess) {
        cudaGetLastError();
        free_dev(c->d_tiled_off);
        free_dev(c->d_tiled_entries);
        return fail(c, LBM_ENOMEM, "lbm_step: cannot allocate the tiles' source-cell lists");
    }
    CUDA_TRY(c, cudaMemcpy(c->d_tiled_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_tiled_entries, list.data(), sizeof(int2) * list.size(), cudaMemcpyHostToDevice));
    c->tiled_version = c->sources_version;
    return LBM_OK;
}

// Planes per block: enough blocks for about 16 waves of the resident ones, and at least 8 planes.
// Each chunk steps two extra planes of the extended tile, but shorter chunks keep neighbouring
// tiles at nearby planes, so that the rows they share are still in L2 (256^3 dipole on GB300, MM:
// 0.714 / 0.705 / 0.693 / 0.691 / 0.701 / 0.715 ms per step at 4 / 8 / 12 / 16 / 24 / 32 waves).
int tiled_chunk(const lbm_ctx* c) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        cudaGetLastError();
    const int occ = std::max(1, c->model == LBM_MM ? mm_tile2_occupancy(c->storage, c->media_mode)
                                                   : hv_tile2_occupancy(c->storage, c->media_mode));
    const long long tiles = (long long)tiled_tiles_x(c) * tiled_tiles_y(c);
    const long long want = (16LL * sms * occ + tiles - 1) / tiles;  // chunks per tile column
    const int chunk = (int)((c->g.nz + want - 1) / want);
    return std::min(c->g.nz, std::max(8, chunk));
}

int tiled_pass(lbm_ctx* c) {
    const int in = c->cur, out = 1 - c->cur;
    StepArgs aA = base_args(c), aB = base_args(c);
    bind_buffers(c, aA, in, out);
    bind_buffers(c, aB, in, out);
    fill_scalars(c, aA, c->t + 1);
    fill_scalars(c, aB, c->t + 2);
    TileArgs T;
    T.tiles_x = tiled_tiles_x(c);
    T.tiles_y = tiled_tiles_y(c);
    T.chunk = tiled_chunk(c);
    T.entry_off = c->d_tiled_off;
    T.entries = c->d_tiled_entries;
    const int launched = c->model == LBM_MM ? mm_launch_tile2(aA, aB, T, c->stream) : hv_launch_tile2(aA, aB, T, c->stream);
    int rc = check_launch(c, launched);
    if (rc != LBM_OK) return rc;
    c->cur = out;
    c->t += 2;
    return LBM_OK;
}

void free_sources_device(lbm_ctx* c) {
    c->sources_version += 1;
    c->h_cell.clear();
    free_dev(c->d_cell);
    free_dev(c->d_entry_begin);
    free_dev(c->d_entry_src);
    free_dev(c->d_entry_w);
    free_dev(c->d_impose_mask);
    free_dev(c->d_block_begin);
    c->n_special = 0;
}

int ensure_partials(lbm_ctx* c, int blocks) {
    if (blocks <= c->partial_capacity) return LBM_OK;
    free_dev(c->d_partials);
    c->partial_capacity = 0;
    if (cudaMalloc(&c->d_partials, sizeof(double) * 3 * (size_t)blocks) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LBM_ENOMEM, "cannot allocate %d reduction partials", blocks);
    }
    c->partial_capacity = blocks;
    return LBM_OK;
}

// Merge every source into one sorted list of special cells with CSR current entries and an
// imposing-source bitmask, and upload it.
int rebuild_sources(lbm_ctx* c) {
    free_sources_device(c);
    std::map<int, std::pair<std::vector<std::pair<int, int>>, uint32_t>> cells;  // cell -> (entries, mask)
    for (size_t k = 0; k < c->sources.size(); ++k) {
        const HostSource& s = c->sources[k];
        for (size_t m = 0; m < s.cells.size(); ++m) {
            auto& slot = cells[s.cells[m]];
            if (s.kind == LBM_SRC_CURRENT) slot.first.emplace_back((int)k, (int)m);
            else slot.second |= (1u << k);
        }
    }
    if (cells.empty()) return LBM_OK;
    std::vector<int> cell, begin, src;
    std::vector<float> w;
    std::vector<uint32_t> mask;
    begin.push_back(0);
    for (auto& kv : cells) {
        cell.push_back(kv.first);
        for (auto& e : kv.second.first) {
            src.push_back(e.first);
            const HostSource& s = c->sources[(size_t)e.first];
            for (int q = 0; q < 3; ++q) w.push_back(s.w[3 * (size_t)e.second + q]);
        }
        begin.push_back((int)src.size());
        mask.push_back(kv.second.second);
    }
    const int ns = (int)cell.size();
    const size_t ne = std::max<size_t>(src.size(), 1);
    if (cudaMalloc(&c->d_cell, sizeof(int) * ns) != cudaSuccess ||
        cudaMalloc(&c->d_entry_begin, sizeof(int) * (ns + 1)) != cudaSuccess ||
        cudaMalloc(&c->d_entry_src, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&c->d_entry_w, sizeof(float) * 3 * ne) != cudaSuccess ||
        cudaMalloc(&c->d_impose_mask, sizeof(uint32_t) * ns) != cudaSuccess) {
        cudaGetLastError();
        free_sources_device(c);
        return fail(c, LBM_ENOMEM, "cannot allocate the source-cell list (%d cells)", ns);
    }
    CUDA_TRY(c, cudaMemcpy(c->d_cell, cell.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_entry_begin, begin.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
    if (!src.empty()) {
        CUDA_TRY(c, cudaMemcpy(c->d_entry_src, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_entry_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(c, cudaMemcpy(c->d_impose_mask, mask.data(), sizeof(uint32_t) * ns, cudaMemcpyHostToDevice));
    // where each block of kBlock cells of the step range starts in the sorted list: a step launch
    // recomputes a block's source cells at the end of the block
    const int r0 = c->z_ghost ? c->g.nx * c->g.ny : 0, r1 = c->z_ghost ? c->g.n - c->g.nx * c->g.ny : c->g.n;
    const int nb = (r1 - r0 + kBlock - 1) / kBlock;
    std::vector<int> bb((size_t)nb + 1);
    for (int b = 0, k = 0; b <= nb; ++b) {
        const long long start = std::min<long long>((long long)r0 + (long long)b * kBlock, r1);
        while (k < ns && cell[(size_t)k] < start) ++k;
        bb[(size_t)b] = k;
    }
    if (cudaMalloc(&c->d_block_begin, sizeof(int) * bb.size()) != cudaSuccess) {
        cudaGetLastError();
        c->d_block_begin = nullptr;
        return fail(c, LBM_ENOMEM, "cannot allocate the blocks' source-cell offsets");
    }
    CUDA_TRY(c, cudaMemcpy(c->d_block_begin, bb.data(), sizeof(int) * bb.size(), cudaMemcpyHostToDevice));
    c->n_special = ns;
    c->h_cell = cell;
    return LBM_OK;
}

// Copy a (possibly device) float array of n values to the host.
int fetch_host(lbm_ctx* c, const float* p, int on_device, int64_t n, std::vector<float>& out) {
    out.resize((size_t)n);
    if (on_device) CUDA_TRY(c, cudaMemcpy(out.data(), p, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
    else memcpy(out.data(), p, sizeof(float) * (size_t)n);
    return LBM_OK;
}

// Coefficients of one material (see MatCoef). Reciprocals used by div_rn are RN(1/d) of the
// stored float d, computed as a float division.
MatCoef coef_for(const lbm_ctx* c, float er, float mr, float sg) {
    MatCoef k;
    if (c->model == LBM_MM) {
        const double g = 1.0 / (1.0 + c->mu0 * (double)sg / (4.0 * (double)er));
        k.c0 = make_float4(er, 1.0f / er, (float)g, (float)(0.25 / (double)mr));
        k.c1 = make_float4(sg, mr, 0.f, 0.f);
    } else {
        const float eps = (float)(c->eps0 * (double)er), mu = (float)(c->mu0 * (double)mr);
        k.c0 = make_float4(eps, 1.0f / eps, mu, 1.0f / mu);
        k.c1 = make_float4(sg, er, 0.f, 0.f);
    }
    return k;
}

// Magic multiplier for division by d of indices below 2^31: k = ceil(log2 d), M = ceil(2^(32+k) / d).
void magic_for(int d, unsigned long long* M, int* k) {
    int kk = 0;
    while ((1LL << kk) < (long long)d) ++kk;
    const unsigned __int128 num = (unsigned __int128)1 << (32 + kk);
    *M = (unsigned long long)((num + (unsigned)d - 1) / (unsigned)d);
    *k = kk;
}

int setup_media(lbm_ctx* c, const lbm_media* m) {
    const int64_t n = c->g.n;
    if (!m || (!m->eps_r && !m->mu_r && !m->sigma)) {
        c->media_mode = kUniform;
        c->uniform = coef_for(c, 1.f, 1.f, 0.f);
        return LBM_OK;
    }
    std::vector<float> er, mr, sg;
    int rc;
    if (m->eps_r && (rc = fetch_host(c, m->eps_r, m->on_device, n, er)) != LBM_OK) return rc;
    if (m->mu_r && (rc = fetch_host(c, m->mu_r, m->on_device, n, mr)) != LBM_OK) return rc;
    if (m->sigma && (rc = fetch_host(c, m->sigma, m->on_device, n, sg)) != LBM_OK) return rc;
    auto val = [&](const std::vector<float>& v, int64_t i, float dflt) { return v.empty() ? dflt : v[(size_t)i]; };
    std::map<std::tuple<float, float, float>, int> ids;
    std::vector<uint8_t> id((size_t)n);
    bool table_ok = true;
    for (int64_t i = 0; i < n; ++i) {
        const float e = val(er, i, 1.f), u = val(mr, i, 1.f), s = val(sg, i, 0.f);
        if (!(std::isfinite(e) && e > 0.f) || !(std::isfinite(u) && u > 0.f) || !(std::isfinite(s) && s >= 0.f))
            return fail(c, LBM_EINVAL, "cell %lld: need finite eps_r > 0, mu_r > 0, sigma >= 0 (got %g, %g, %g)",
                        (long long)i, e, u, s);
        if (!table_ok) continue;
        auto key = std::make_tuple(e, u, s);
        auto it = ids.find(key);
        if (it == ids.end()) {
            if (ids.size() == 256) {
                table_ok = false;
                continue;
            }
            it = ids.emplace(key, (int)ids.size()).first;
        }
        id[(size_t)i] = (uint8_t)it->second;
    }
    if (table_ok && ids.size() == 1) {
        auto key = ids.begin()->first;
        c->media_mode = kUniform;
        c->uniform = coef_for(c, std::get<0>(key), std::get<1>(key), std::get<2>(key));
        return LBM_OK;
    }
    if (table_ok) {
        std::vector<MatCoef> table(ids.size());
        for (auto& kv : ids)
            table[(size_t)kv.second] = coef_for(c, std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first));
        if (cudaMalloc(&c->mat_id, (size_t)n) != cudaSuccess ||
            cudaMalloc(&c->mat_table, sizeof(MatCoef) * table.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LBM_ENOMEM, "cannot allocate the material table");
        }
        CUDA_TRY(c, cudaMemcpy(c->mat_id, id.data(), (size_t)n, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->mat_table, table.data(), sizeof(MatCoef) * table.size(), cudaMemcpyHostToDevice));
        c->media_mode = kTable;
        return LBM_OK;
    }
    c->media_mode = kPerCell;
    float** dst[3] = {&c->eps_r, &c->mu_r, &c->sigma};
    const std::vector<float>* srcv[3] = {&er, &mr, &sg};
    const float dflt[3] = {1.f, 1.f, 0.f};
    for (int q = 0; q < 3; ++q) {
        if (cudaMalloc(dst[q], sizeof(float) * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LBM_ENOMEM, "cannot allocate per-cell media");
        }
        std::vector<float> v = srcv[q]->empty() ? std::vector<float>((size_t)n, dflt[q]) : *srcv[q];
        CUDA_TRY(c, cudaMemcpy(*dst[q], v.data(), sizeof(float) * (size_t)n, cudaMemcpyHostToDevice));
    }
    return LBM_OK;
}

void release(lbm_ctx* c) {
    for (int b = 0; b < 2; ++b) {
        free_dev(c->buf[b]);
        free_dev(c->buf2[b]);
        free_dev(c->rho[b]);
    }
    free_dev(c->rest1);
    free_dev(c->mat_id);
    free_dev(c->mat_table);
    free_dev(c->eps_r);
    free_dev(c->mu_r);
    free_dev(c->sigma);
    free_sources_device(c);
    free_dev(c->d_partials);
    free_dev(c->d_result);
    free_dev(c->adj_ws);
    c->adj_ws_bytes = 0;
    free_dev(c->host_stage);
    c->host_stage_bytes = 0;
    free_dev(c->halo_stage);
    c->halo_stage_bytes = 0;
    free_dev(c->fused_planes);
    c->fused_planes_bytes = 0;
    free_dev(c->fused_ctrl);
    free_dev(c->d_tile_special);
    free_dev(c->d_tiled_off);
    free_dev(c->d_tiled_entries);
}

// The context's device staging buffer for host fields, at least `bytes` long. It is kept between
// calls (a per-call cudaMalloc / cudaFree pair, with the device-wide wait of cudaFree, cost more
// than the copy itself) and grown when a call needs more. The caller has waited for the stream's
// earlier use of it: every host-side call that uses it waits before returning.
int host_staging(lbm_ctx* c, size_t bytes, float** dev) {
    if (c->host_stage_bytes < bytes) {
        free_dev(c->host_stage);
        c->host_stage_bytes = 0;
        if (cudaMalloc(&c->host_stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->host_stage = nullptr;
            return fail(c, LBM_ENOMEM, "cannot allocate a staging buffer of %zu bytes", bytes);
        }
        c->host_stage_bytes = bytes;
    }
    *dev = c->host_stage;
    return LBM_OK;
}

// Copy a 3 x n (or k x n) input to a device staging buffer when it is on the host.
int stage_input(lbm_ctx* c, const float* p, int on_device, size_t count, float** dev, bool* owned) {
    if (on_device) {
        *dev = const_cast<float*>(p);
        *owned = false;
        return LBM_OK;
    }
    if (cudaMalloc(dev, sizeof(float) * count) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LBM_ENOMEM, "cannot allocate a staging buffer of %zu floats", count);
    }
    *owned = true;
    CUDA_TRY(c, cudaMemcpyAsync(*dev, p, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_num_populations(int model) { return model == LBM_MM ? 50 : (model == LBM_HV ? 36 : LBM_EINVAL); }

int lbm_create(int model, int nx, int ny, int nz, const lbm_media* media, const lbm_options* opts, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    if (model != LBM_MM && model != LBM_HV) return fail(nullptr, LBM_EINVAL, "lbm_create: unknown model %d", model);
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "lbm_create: dimensions must be >= 1");
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > (int64_t)INT32_MAX) return fail(nullptr, LBM_EINVAL, "lbm_create: %lld cells exceed 2^31 - 1", (long long)n);
    const int storage = opts ? opts->storage : LBM_F32;
    if (storage != LBM_F32 && storage != LBM_BF16 && storage != LBM_F16 && storage != LBM_F24)
        return fail(nullptr, LBM_EINVAL, "lbm_create: unknown storage %d", storage);
    double scale = (opts && storage != LBM_F32) ? opts->storage_scale : 0.0;
    if (scale == 0.0) scale = 1.0;
    int scale_exp = 0;
    if (!(scale > 0) || !std::isfinite(scale) || std::frexp(scale, &scale_exp) != 0.5 || scale_exp < -100 ||
        scale_exp > 100)
        return fail(nullptr, LBM_EINVAL, "lbm_create: storage_scale must be a power of two in [2^-100, 2^100]");
    const int z_ghost = opts ? opts->z_ghost : 0;
    if (z_ghost != 0 && z_ghost != 1) return fail(nullptr, LBM_EINVAL, "lbm_create: z_ghost must be 0 or 1");
    if (z_ghost && nz < 3) return fail(nullptr, LBM_EINVAL, "lbm_create: a z_ghost slab needs nz >= 3");
    if (z_ghost && storage == LBM_F24)
        return fail(nullptr, LBM_EUNSUPPORTED, "lbm_create: z_ghost slabs do not take LBM_F24 storage");
    double eps0 = opts ? opts->eps0 : 0.0, mu0 = opts ? opts->mu0 : 0.0;
    if (eps0 < 0 || mu0 < 0 || !std::isfinite(eps0) || !std::isfinite(mu0))
        return fail(nullptr, LBM_EINVAL, "lbm_create: eps0, mu0 must be >= 0");
    if (model == LBM_MM) {
        if ((eps0 != 0 && eps0 != 1.0) || (mu0 != 0 && mu0 != 2.0))
            return fail(nullptr, LBM_EUNSUPPORTED, "lbm_create: the MM model fixes eps0 = 1, mu0 = 2");
        eps0 = 1.0;
        mu0 = 2.0;
    } else {
        if (eps0 == 0) eps0 = 3.0;
        if (mu0 == 0) mu0 = 3.0;
    }
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "lbm_create: out of host memory");
    c->model = model;
    c->g = Geometry{nx, ny, nz, (int)n, 0, 0, 0, 0};
    magic_for(nx, &c->g.mx, &c->g.kx);
    magic_for(nx * ny, &c->g.mxy, &c->g.kxy);
    c->stream = opts ? static_cast<cudaStream_t>(opts->cuda_stream) : nullptr;
    c->track_rho = (opts && opts->track_rho && model == LBM_MM) ? 1 : 0;
    c->z_ghost = z_ghost;
    c->eps0 = eps0;
    c->mu0 = mu0;
    c->storage = storage;
    c->scale = (float)scale;
    int rc;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, LBM_ECUDA, "lbm_create: no CUDA device");
    }
    const size_t pop_bytes = group_bytes(model, storage) * (size_t)n;
    const size_t pop2_bytes = pair_bytes(storage) * (size_t)n;
    for (int b = 0; b < 2; ++b) {
        bool ok = cudaMalloc(&c->buf[b], pop_bytes) == cudaSuccess;
        if (ok && model == LBM_HV) ok = cudaMalloc(&c->buf2[b], pop2_bytes) == cudaSuccess;
        if (ok && c->track_rho) ok = cudaMalloc(&c->rho[b], sizeof(float) * (size_t)n) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            release(c);
            delete c;
            return fail(nullptr, LBM_ENOMEM, "lbm_create: cannot allocate populations for %lld cells", (long long)n);
        }
    }
    if (c->track_rho && cudaMalloc(&c->rest1, sizeof(float) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        delete c;
        return fail(nullptr, LBM_ENOMEM, "lbm_create: cannot allocate rest populations");
    }
    if ((rc = setup_media(c, media)) != LBM_OK) {
        g_create_error = c->err;
        release(c);
        delete c;
        return rc;
    }
    c->reduce_blocks = std::max(1, std::min((int)((n + kBlock - 1) / kBlock), 152 * 4));
    if (cudaMalloc(&c->d_result, sizeof(double) * 3) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        delete c;
        return fail(nullptr, LBM_ENOMEM, "lbm_create: cannot allocate reduction result");
    }
    bool zero_ok = true;
    for (int b = 0; b < 2; ++b) {
        zero_ok &= cudaMemsetAsync(c->buf[b], 0, pop_bytes, c->stream) == cudaSuccess;
        if (c->buf2[b]) zero_ok &= cudaMemsetAsync(c->buf2[b], 0, pop2_bytes, c->stream) == cudaSuccess;
        if (c->rho[b]) zero_ok &= cudaMemsetAsync(c->rho[b], 0, sizeof(float) * (size_t)n, c->stream) == cudaSuccess;
    }
    if (c->rest1) zero_ok &= cudaMemsetAsync(c->rest1, 0, sizeof(float) * (size_t)n, c->stream) == cudaSuccess;
    if (!zero_ok) {
        cudaError_t e = cudaGetLastError();
        release(c);
        delete c;
        return fail(nullptr, LBM_ECUDA, "lbm_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return LBM_OK;
    ensure_device(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    release(ctx);
    delete ctx;
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* ctx, const float* E, const float* B, int on_device) {
    if (!ctx) return LBM_EINVAL;
    if (!E || !B) return fail(ctx, LBM_EINVAL, "lbm_init_fields: E and B are required");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    const size_t cnt = 3 * (size_t)ctx->g.n;
    const float *dE = E, *dB = B;
    if (!on_device) {
        float* st = nullptr;
        if ((rc = host_staging(ctx, 2 * cnt * sizeof(float), &st)) != LBM_OK) return rc;
        CUDA_TRY(ctx, cudaMemcpyAsync(st, E, sizeof(float) * cnt, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(st + cnt, B, sizeof(float) * cnt, cudaMemcpyHostToDevice, ctx->stream));
        dE = st;
        dB = st + cnt;
    }
    StepArgs a = base_args(ctx);
    ctx->cur = 0;
    bind_buffers(ctx, a, 1, 0);
    const int launched = ctx->model == LBM_MM ? mm_launch_init(a, dE, dB, ctx->stream) : hv_launch_init(a, dE, dB, ctx->stream);
    rc = check_launch(ctx, launched);
    if (rc == LBM_OK && ctx->rho[0]) {
        if (cudaMemsetAsync(ctx->rho[0], 0, sizeof(float) * ctx->g.n, ctx->stream) != cudaSuccess ||
            cudaMemsetAsync(ctx->rest1, 0, sizeof(float) * ctx->g.n, ctx->stream) != cudaSuccess)
            rc = fail(ctx, LBM_ECUDA, "lbm_init_fields: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (!on_device && cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == LBM_OK)  // the caller may reuse E, B
        rc = fail(ctx, LBM_ECUDA, "lbm_init_fields: %s", cudaGetErrorString(cudaGetLastError()));
    ctx->t = 0;
    return rc;
}

int lbm_set_source(lbm_ctx* ctx, const lbm_source* src) {
    if (!ctx) return LBM_EINVAL;
    if (!src) return fail(ctx, LBM_EINVAL, "lbm_set_source: src is NULL");
    if ((int)ctx->sources.size() >= LBM_MAX_SOURCES)
        return fail(ctx, LBM_EINVAL, "lbm_set_source: at most %d sources", LBM_MAX_SOURCES);
    if (src->kind != LBM_SRC_CURRENT && src->kind != LBM_SRC_IMPOSE)
        return fail(ctx, LBM_EINVAL, "lbm_set_source: unknown kind %d", src->kind);
    if (src->n_cells < 0 || (src->n_cells > 0 && !src->cells))
        return fail(ctx, LBM_EINVAL, "lbm_set_source: bad cell list");
    if (src->kind == LBM_SRC_CURRENT && src->n_cells > 0 && !src->w)
        return fail(ctx, LBM_EINVAL, "lbm_set_source: a current source needs weights");
    const lbm_time_fn& fn = src->fn;
    if (fn.kind != LBM_FN_SIN && fn.kind != LBM_FN_TABLE && fn.kind != LBM_FN_CONST)
        return fail(ctx, LBM_EINVAL, "lbm_set_source: unknown time function %d", fn.kind);
    if (fn.kind == LBM_FN_SIN && !(fn.period != 0.0 && std::isfinite(fn.period)))
        return fail(ctx, LBM_EINVAL, "lbm_set_source: sin period must be finite and non-zero");
    if (fn.kind == LBM_FN_TABLE && (fn.table_len < 0 || (fn.table_len > 0 && !fn.table)))
        return fail(ctx, LBM_EINVAL, "lbm_set_source: bad table");
    HostSource s;
    s.kind = src->kind;
    s.cells.resize((size_t)src->n_cells);
    for (int64_t m = 0; m < src->n_cells; ++m) {
        if (src->cells[m] < 0 || src->cells[m] >= ctx->g.n)
            return fail(ctx, LBM_EINVAL, "lbm_set_source: cell %lld out of range", (long long)src->cells[m]);
        const int64_t plane = src->cells[m] / ((int64_t)ctx->g.nx * ctx->g.ny);
        if (ctx->z_ghost && (plane == 0 || plane == ctx->g.nz - 1))
            return fail(ctx, LBM_EINVAL, "lbm_set_source: cell %lld lies in a ghost plane", (long long)src->cells[m]);
        s.cells[(size_t)m] = (int)src->cells[m];
    }
    if (src->kind == LBM_SRC_CURRENT) s.w.assign(src->w, src->w + 3 * src->n_cells);
    for (int q = 0; q < 3; ++q) {
        s.E0[q] = src->kind == LBM_SRC_IMPOSE ? src->E0[q] : 0.f;
        s.B0[q] = src->kind == LBM_SRC_IMPOSE ? src->B0[q] : 0.f;
    }
    s.fn = fn;
    s.fn.table = nullptr;
    if (fn.kind == LBM_FN_TABLE && fn.table_len > 0) s.table.assign(fn.table, fn.table + fn.table_len);
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    CUDA_TRY(ctx, ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    ctx->sources.push_back(std::move(s));
    rc = rebuild_sources(ctx);
    if (rc != LBM_OK) ctx->sources.pop_back();
    return rc;
}

int lbm_clear_sources(lbm_ctx* ctx) {
    if (!ctx) return LBM_EINVAL;
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    CUDA_TRY(ctx, ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    ctx->sources.clear();
    free_sources_device(ctx);
    return LBM_OK;
}

int lbm_step(lbm_ctx* ctx, int n) {
    if (!ctx) return LBM_EINVAL;
    if (n < 0) return fail(ctx, LBM_EINVAL, "lbm_step: n must be >= 0");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    int s = 0;
    const int kind = n >= 2 ? pass_kind(ctx) : kPassNone;
    if (kind == kPassRing) {
        if ((rc = ensure_fused(ctx)) != LBM_OK) return rc;
        for (; s + 2 <= n; s += 2)
            if ((rc = fused_pass(ctx)) != LBM_OK) return rc;
    } else if (kind == kPassTiled) {
        if ((rc = ensure_tiled(ctx)) != LBM_OK) return rc;
        for (; s + 2 <= n; s += 2)
            if ((rc = tiled_pass(ctx)) != LBM_OK) return rc;
    }
    StepArgs a = base_args(ctx);
    for (; s < n; ++s) {
        const int in = ctx->cur, out = 1 - ctx->cur;
        bind_buffers(ctx, a, in, out);
        fill_scalars(ctx, a, ctx->t + 1);
        const int launched = ctx->model == LBM_MM ? mm_launch_step(a, ctx->stream) : hv_launch_step(a, ctx->stream);
        if ((rc = check_launch(ctx, launched)) != LBM_OK) return rc;
        ctx->cur = out;
        ctx->t += 1;
    }
    return LBM_OK;
}

int lbm_fields(lbm_ctx* ctx, unsigned mask, float* out, int on_device) {
    if (!ctx) return LBM_EINVAL;
    if (!out) return fail(ctx, LBM_EINVAL, "lbm_fields: out is NULL");
    if (mask == 0 || (mask & ~31u)) return fail(ctx, LBM_EINVAL, "lbm_fields: bad mask 0x%x", mask);
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    if (!on_device && (rc = check_fused_abort(ctx)) != LBM_OK) return rc;
    int nf = 0;
    for (int b = 0; b < 5; ++b) nf += (mask >> b) & 1;
    const size_t cnt = 3 * (size_t)ctx->g.n * nf;
    float* dev = out;
    if (!on_device && (rc = host_staging(ctx, sizeof(float) * cnt, &dev)) != LBM_OK) return rc;
    FieldsOut fo{nullptr, nullptr, nullptr, nullptr, nullptr};
    float** slots[5] = {&fo.E, &fo.B, &fo.D, &fo.H, &fo.J};
    size_t off = 0;
    for (int b = 0; b < 5; ++b)
        if ((mask >> b) & 1) {
            *slots[b] = dev + off;
            off += 3 * (size_t)ctx->g.n;
        }
    StepArgs a = base_args(ctx);
    bind_buffers(ctx, a, ctx->cur, 1 - ctx->cur);
    fill_scalars(ctx, a, ctx->t + 1);
    const int launched = ctx->model == LBM_MM ? mm_launch_fields(a, fo, ctx->stream) : hv_launch_fields(a, fo, ctx->stream);
    rc = check_launch(ctx, launched);
    if (!on_device) {
        if (rc == LBM_OK && cudaMemcpyAsync(out, dev, sizeof(float) * cnt, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            rc = fail(ctx, LBM_ECUDA, "lbm_fields: copy: %s", cudaGetErrorString(cudaGetLastError()));
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == LBM_OK)
            rc = fail(ctx, LBM_ECUDA, "lbm_fields: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return rc;
}

int lbm_get_populations(lbm_ctx* ctx, float* out, int on_device) {
    if (!ctx) return LBM_EINVAL;
    if (!out) return fail(ctx, LBM_EINVAL, "lbm_get_populations: out is NULL");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    if (!on_device && (rc = check_fused_abort(ctx)) != LBM_OK) return rc;
    const size_t cnt = (size_t)lbm_num_populations(ctx->model) * ctx->g.n;
    float* dev = out;
    if (!on_device && cudaMalloc(&dev, sizeof(float) * cnt) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LBM_ENOMEM, "lbm_get_populations: cannot allocate %zu floats", cnt);
    }
    StepArgs a = base_args(ctx);
    bind_buffers(ctx, a, ctx->cur, 1 - ctx->cur);
    const int launched = ctx->model == LBM_MM ? mm_launch_get(a, dev, ctx->stream) : hv_launch_get(a, dev, ctx->stream);
    rc = check_launch(ctx, launched);
    if (!on_device) {
        if (rc == LBM_OK && cudaMemcpyAsync(out, dev, sizeof(float) * cnt, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            rc = fail(ctx, LBM_ECUDA, "lbm_get_populations: copy: %s", cudaGetErrorString(cudaGetLastError()));
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == LBM_OK)
            rc = fail(ctx, LBM_ECUDA, "lbm_get_populations: %s", cudaGetErrorString(cudaGetLastError()));
        cudaFree(dev);
    }
    return rc;
}

int lbm_set_populations(lbm_ctx* ctx, const float* in, int on_device, int64_t t) {
    if (!ctx) return LBM_EINVAL;
    if (!in) return fail(ctx, LBM_EINVAL, "lbm_set_populations: in is NULL");
    if (t < 0) return fail(ctx, LBM_EINVAL, "lbm_set_populations: t must be >= 0");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    const size_t cnt = (size_t)lbm_num_populations(ctx->model) * ctx->g.n;
    float* dev = nullptr;
    bool owned = false;
    if ((rc = stage_input(ctx, in, on_device, cnt, &dev, &owned)) != LBM_OK) return rc;
    StepArgs a = base_args(ctx);
    ctx->cur = 0;
    bind_buffers(ctx, a, 1, 0);
    const int launched = ctx->model == LBM_MM ? mm_launch_set(a, dev, ctx->stream) : hv_launch_set(a, dev, ctx->stream);
    rc = check_launch(ctx, launched);
    if (owned) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(dev);
    }
    ctx->t = t;
    return rc;
}

int lbm_reduce(lbm_ctx* ctx, double out[3]) {
    if (!ctx) return LBM_EINVAL;
    if (!out) return fail(ctx, LBM_EINVAL, "lbm_reduce: out is NULL");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    if ((rc = check_fused_abort(ctx)) != LBM_OK) return rc;
    const int ns_blocks = ctx->n_special > 0 ? (ctx->n_special + kBlock - 1) / kBlock : 0;
    if ((rc = ensure_partials(ctx, ctx->reduce_blocks + ns_blocks)) != LBM_OK) return rc;
    StepArgs a = base_args(ctx);
    bind_buffers(ctx, a, ctx->cur, 1 - ctx->cur);
    fill_scalars(ctx, a, ctx->t + 1);
    const int launched = ctx->model == LBM_MM
                             ? mm_launch_reduce(a, ctx->d_partials, ctx->reduce_blocks, ctx->d_result, ctx->stream)
                             : hv_launch_reduce(a, ctx->d_partials, ctx->reduce_blocks, ctx->d_result, ctx->stream);
    if ((rc = check_launch(ctx, launched)) != LBM_OK) return rc;
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->d_result, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_check_finite(lbm_ctx* ctx) {
    double r[3];
    int rc = lbm_reduce(ctx, r);
    if (rc != LBM_OK) return rc;
    if (!std::isfinite(r[1])) return fail(ctx, LBM_ENONFINITE, "non-finite population (sum of squares %g)", r[1]);
    return LBM_OK;
}

int64_t lbm_time(const lbm_ctx* ctx) { return ctx ? ctx->t : -1; }
int64_t lbm_launch_count(const lbm_ctx* ctx) { return ctx ? ctx->launches : -1; }

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int lbm_sync(lbm_ctx* ctx) {
    if (!ctx) return LBM_EINVAL;
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return check_fused_abort(ctx);
}

int lbm_set_step_fusion(lbm_ctx* ctx, int mode, int tile_cells) {
    if (!ctx) return LBM_EINVAL;
    if (mode < 0 || mode > 3) return fail(ctx, LBM_EINVAL, "lbm_set_step_fusion: mode must be 0, 1, 2 or 3");
    if (tile_cells < 0 || tile_cells % kBlock != 0 || tile_cells > 16 * kBlock)
        return fail(ctx, LBM_EINVAL, "lbm_set_step_fusion: tile_cells must be 0 or a multiple of %d up to %d", kBlock,
                    16 * kBlock);
    if (tile_cells != 0 && tile_cells != fused_tile_cells(ctx)) {
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        else cudaDeviceSynchronize();
        free_dev(ctx->fused_ctrl);  // its flag array depends on the tile count
        ctx->tile_special_version = -1;  // so do the tiles' source-cell offsets
        ctx->fused_tile = tile_cells;
    }
    ctx->fusion = mode;
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* ctx, long long ns) {
    if (!ctx) return LBM_EINVAL;
    ctx->wait_limit_ns = ns;
    return LBM_OK;
}

int lbm_step_fusion_active(lbm_ctx* ctx) {
    if (!ctx) return LBM_EINVAL;
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    return pass_kind(ctx);
}

}  // extern "C"

// Deterministic final reduction: one block, each thread sums a fixed strided subset in order.
namespace lbm {
namespace {
__global__ void __launch_bounds__(kBlock) reduce_partials_kernel(const double* __restrict__ p, int nb,
                                                                 double* __restrict__ result) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += kBlock) {
        s0 += p[3 * b];
        s1 += p[3 * b + 1];
        s2 += p[3 * b + 2];
    }
    block_sum3_store(s0, s1, s2, result);
}
}  // namespace

int launch_reduce_partials(const double* partials, int n_blocks, double* result, cudaStream_t st) {
    reduce_partials_kernel<<<1, kBlock, 0, st>>>(partials, n_blocks, result);
    return 1;
}

namespace {
__global__ void __launch_bounds__(kBlock) sum_doubles_kernel(const double* __restrict__ v, int count,
                                                             double* __restrict__ result) {
    double s = 0.0;
    for (int k = threadIdx.x; k < count; k += kBlock) s += v[k];
    block_sum3_store(s, 0.0, 0.0, result);
}
}  // namespace

int launch_sum_doubles(const double* v, int count, double* result, cudaStream_t st) {
    sum_doubles_kernel<<<1, kBlock, 0, st>>>(v, count, result);
    return 1;
}

namespace {
// blockIdx.y selects the chunk; blocks stride over its words. W is the widest of 16, 8, 4 bytes that
// divides both addresses and the size (decided on the host, the same for every block of a chunk).
template <typename W>
__device__ __forceinline__ void copy_words(const HaloChunk& c) {
    const W* __restrict__ src = reinterpret_cast<const W*>(c.src);
    W* __restrict__ dst = reinterpret_cast<W*>(c.dst);
    const long long words = c.bytes / (long long)sizeof(W);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < words;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

__global__ void __launch_bounds__(kBlock) halo_copy_kernel(HaloCopy h) {
    const HaloChunk& c = h.c[blockIdx.y];
    if (c.width == 16) copy_words<uint4>(c);
    else if (c.width == 8) copy_words<uint2>(c);
    else copy_words<unsigned>(c);
}
}  // namespace

int launch_halo_copy(HaloCopy h, cudaStream_t st) {
    if (h.count <= 0) return 0;
    long long most = 0;
    for (int k = 0; k < h.count; ++k) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(h.c[k].src) | reinterpret_cast<uintptr_t>(h.c[k].dst) |
                            (uintptr_t)h.c[k].bytes;
        h.c[k].width = (a % 16 == 0) ? 16 : (a % 8 == 0 ? 8 : 4);
        most = std::max(most, h.c[k].bytes / h.c[k].width);
    }
    const int bx = (int)std::max<long long>(1, std::min<long long>((most + kBlock - 1) / kBlock, 152 * 4));
    halo_copy_kernel<<<dim3(bx, h.count), kBlock, 0, st>>>(h);
    return 1;
}
}  // namespace lbm

// ------------------------------------------------------------------------------------------------
// lbm_reduce_noalloc: the reductions of lbm_reduce without any device allocation.
//
// lbm_reduce keeps its per-block partial sums in device memory that it allocates on first use (and
// again when the source-cell list grows). Some callers cannot allow that: their device memory is
// owned by a pool of their own that must account for every byte, or their stepping loop cannot take
// the implicit device synchronisation of cudaMalloc/cudaFree. This entry point runs the same kernels
// with the partial sums in the file-scope array below instead. Every GPU that loads the library
// holds the array (about 96 KiB) until the process exits.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr int kStaticPartialBlocks = 4096;  // partial-sum slots (3 doubles each); the size limit

static __device__ __align__(256) double g_reduce_scratch[3 * kStaticPartialBlocks + 3];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_reduce_scratch on the current device, looked up once per device. In host
// code the array's name is only a host-side stand-in, never a device address.
int static_scratch(lbm_ctx* ctx, double** out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(ctx, LBM_EUNSUPPORTED, "lbm_reduce_noalloc: device %d beyond the %d supported", ctx->device,
                    kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_reduce_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, LBM_ECUDA, "lbm_reduce_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[ctx->device] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[ctx->device];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_noalloc(lbm_ctx* ctx, double* out, int on_device) {
    if (!ctx) return LBM_EINVAL;
    if (!out) return fail(ctx, LBM_EINVAL, "lbm_reduce_noalloc: out is NULL");
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    // Host output reports a two-step pass that stopped, as lbm_reduce does; device output is
    // stream-ordered and leaves that to the next waiting call.
    if (!on_device && (rc = check_fused_abort(ctx)) != LBM_OK) return rc;
    // Only the MM reduction keeps one partial per 256 source cells: its energy takes a correction
    // at source cells, where J_ext enters E. HV's E does not depend on J_ext, so it needs the
    // lattice's blocks alone.
    const int ns_blocks =
        ctx->model == LBM_MM && ctx->n_special > 0 ? (ctx->n_special + kBlock - 1) / kBlock : 0;
    const int needed = ctx->reduce_blocks + ns_blocks;
    if (needed > kStaticPartialBlocks)
        return fail(ctx, LBM_EINVAL,
                    "lbm_reduce_noalloc: needs %d partial-sum slots but the static scratch holds %d "
                    "(%d source cells is more than the %d it allows for this MM lattice)",
                    needed, kStaticPartialBlocks, ctx->n_special, (kStaticPartialBlocks - ctx->reduce_blocks) * kBlock);
    double* scratch = nullptr;
    if ((rc = static_scratch(ctx, &scratch)) != LBM_OK) return rc;
    // Every slot the final sum reads is written by this call's kernels first, so nothing needs
    // clearing; the result lands in the caller's device buffer or in the last 3 slots.
    double* result = on_device ? out : scratch + 3 * kStaticPartialBlocks;
    StepArgs a = base_args(ctx);
    bind_buffers(ctx, a, ctx->cur, 1 - ctx->cur);
    fill_scalars(ctx, a, ctx->t + 1);
    const int launched = ctx->model == LBM_MM
                             ? mm_launch_reduce(a, scratch, ctx->reduce_blocks, result, ctx->stream)
                             : hv_launch_reduce(a, scratch, ctx->reduce_blocks, result, ctx->stream);
    if ((rc = check_launch(ctx, launched)) != LBM_OK) return rc;
    if (!on_device) {
        CUDA_TRY(ctx, cudaMemcpyAsync(out, result, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBM_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched stepping of several lattices (mesh-refinement sweeps): lbm_batch_*.
// ------------------------------------------------------------------------------------------------
struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    int model = 0, storage = 0, device = 0;
    bool rho = false;
    cudaStream_t stream = nullptr;
    int block = 256;     // threads per block of the main launch
    int persistent = 0;  // 1: grid of resident blocks striding over the tiles
    BatchLattice* d_lat = nullptr;
    BatchTile* d_tiles = nullptr;
    size_t tiles_cap = 0;
    BatchTile* d_stiles = nullptr;
    size_t stiles_cap = 0;
    float* d_stable = nullptr;
    size_t stable_cap = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> graph_key;
    int64_t launches = 0;
    std::string err;
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_error = buf;
    return code;
}

#define BCUDA_TRY(b, call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return bfail((b), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void drop_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_key.clear();
}

template <class T>
int ensure_capacity(lbm_batch* b, T** p, size_t* cap, size_t count) {
    if (count <= *cap) return LBM_OK;
    drop_graph(b);  // a captured graph holds the old address
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LBM_ENOMEM, "batch: cannot allocate %zu entries", count);
    }
    *cap = count;
    return LBM_OK;
}

// Lattice order (decreasing step count, so the active lattices of any step form a prefix), tiles and
// per-step active tile counts for the current block size.
struct BatchPlan {
    std::vector<int> order;
    std::vector<BatchTile> tiles, stiles;
    std::vector<int> tile_end, stile_end;  // cumulative counts per lattice in order
    int max_steps = 0;
};

BatchPlan plan_batch(const lbm_batch* b, const int* steps) {
    BatchPlan p;
    const int count = (int)b->ctx.size();
    p.order.resize(count);
    for (int k = 0; k < count; ++k) p.order[k] = k;
    std::stable_sort(p.order.begin(), p.order.end(), [&](int x, int y) { return steps[x] > steps[y]; });
    for (int k : p.order) {
        const lbm_ctx* c = b->ctx[k];
        for (int begin = 0; begin < c->g.n; begin += b->block) p.tiles.push_back(BatchTile{k, begin});
        for (int begin = 0; begin < c->n_special; begin += kBlock) p.stiles.push_back(BatchTile{k, begin});
        p.tile_end.push_back((int)p.tiles.size());
        p.stile_end.push_back((int)p.stiles.size());
        p.max_steps = std::max(p.max_steps, steps[k]);
    }
    return p;
}

// Number of tiles of the lattices still active at step j (a prefix of the order).
int active_prefix(const BatchPlan& p, const int* steps, int j, const std::vector<int>& ends) {
    int last = -1;
    for (size_t r = 0; r < p.order.size(); ++r)
        if (steps[p.order[r]] > j) last = (int)r;
    return last < 0 ? 0 : ends[(size_t)last];
}

// Upload descriptors (and source tables) for a call advancing lattice k by steps[k].
int upload_batch(lbm_batch* b, const int* steps, int max_steps) {
    const int count = (int)b->ctx.size();
    size_t stable_size = 0;
    for (int k = 0; k < count; ++k) stable_size += b->ctx[k]->sources.size() * (size_t)std::max(max_steps, 1);
    int rc;
    if ((rc = ensure_capacity(b, &b->d_stable, &b->stable_cap, std::max<size_t>(stable_size, 1))) != LBM_OK) return rc;
    std::vector<float> table(std::max<size_t>(stable_size, 1), 0.f);
    std::vector<BatchLattice> lat((size_t)count);
    size_t off = 0;
    for (int k = 0; k < count; ++k) {
        lbm_ctx* c = b->ctx[k];
        BatchLattice& L = lat[(size_t)k];
        memset(&L, 0, sizeof(L));
        L.base = base_args(c);
        for (int q = 0; q < 2; ++q) {
            L.buf[q] = c->buf[q];
            L.buf2[q] = c->model == LBM_HV ? c->buf2[q] : c->rest1;
            L.rho[q] = c->rho[q];
        }
        L.cur0 = c->cur;
        L.steps = steps[k];
        L.n_src = (int)c->sources.size();
        L.s_stride = std::max(max_steps, 1);
        L.s_table = b->d_stable + off;
        for (int s = 0; s < L.n_src; ++s)
            for (int j = 0; j < steps[k]; ++j)
                table[off + (size_t)s * L.s_stride + (size_t)j] = (float)time_value(c->sources[(size_t)s], c->t + 1 + j);
        off += (size_t)L.n_src * L.s_stride;
    }
    BCUDA_TRY(b, cudaMemcpyAsync(b->d_lat, lat.data(), sizeof(BatchLattice) * count, cudaMemcpyHostToDevice, b->stream));
    BCUDA_TRY(b, cudaMemcpyAsync(b->d_stable, table.data(), sizeof(float) * table.size(), cudaMemcpyHostToDevice,
                                 b->stream));
    return LBM_OK;
}

int upload_tiles(lbm_batch* b, const BatchPlan& p) {
    int rc;
    if ((rc = ensure_capacity(b, &b->d_tiles, &b->tiles_cap, std::max<size_t>(p.tiles.size(), 1))) != LBM_OK) return rc;
    if ((rc = ensure_capacity(b, &b->d_stiles, &b->stiles_cap, std::max<size_t>(p.stiles.size(), 1))) != LBM_OK) return rc;
    if (!p.tiles.empty())
        BCUDA_TRY(b, cudaMemcpyAsync(b->d_tiles, p.tiles.data(), sizeof(BatchTile) * p.tiles.size(),
                                     cudaMemcpyHostToDevice, b->stream));
    if (!p.stiles.empty())
        BCUDA_TRY(b, cudaMemcpyAsync(b->d_stiles, p.stiles.data(), sizeof(BatchTile) * p.stiles.size(),
                                     cudaMemcpyHostToDevice, b->stream));
    return LBM_OK;
}

BatchLaunch launch_config(const lbm_batch* b) {
    BatchLaunch L;
    L.lat = b->d_lat;
    L.tiles = b->d_tiles;
    L.stiles = b->d_stiles;
    L.block = b->block;
    L.storage = b->storage;
    L.rho = b->rho;
    L.grid_cap = 0;
    if (b->persistent) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        const int occ = b->model == LBM_MM ? mm_batch_occupancy(b->storage, b->block, b->rho)
                                           : hv_batch_occupancy(b->storage, b->block);
        L.grid_cap = std::max(1, sms * std::max(occ, 1));
    }
    return L;
}

// Enqueue every step of the call on the batch stream.
int enqueue_steps(lbm_batch* b, const BatchPlan& p, const int* steps, int64_t* launched) {
    const BatchLaunch L = launch_config(b);
    for (int j = 0; j < p.max_steps; ++j) {
        const int nt = active_prefix(p, steps, j, p.tile_end);
        const int ns = active_prefix(p, steps, j, p.stile_end);
        *launched += b->model == LBM_MM ? mm_launch_batch_step(L, j, nt, ns, b->stream)
                                        : hv_launch_batch_step(L, j, nt, ns, b->stream);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "batched launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_ctx* const* ctxs, int count, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: out is NULL");
    *out = nullptr;
    if (!ctxs || count < 1) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: need at least one context");
    for (int k = 0; k < count; ++k) {
        if (!ctxs[k]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d is NULL", k);
        if (ctxs[k]->z_ghost)
            return bfail(nullptr, LBM_EUNSUPPORTED, "lbm_batch_create: context %d is a z_ghost slab", k);
        for (int q = 0; q < k; ++q)
            if (ctxs[q] == ctxs[k]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d repeated", k);
        if (ctxs[k]->model != ctxs[0]->model || ctxs[k]->storage != ctxs[0]->storage ||
            ctxs[k]->stream != ctxs[0]->stream || ctxs[k]->device != ctxs[0]->device ||
            (ctxs[k]->rho[0] != nullptr) != (ctxs[0]->rho[0] != nullptr))
            return bfail(nullptr, LBM_EINVAL,
                         "lbm_batch_create: contexts must share model, storage, track_rho, stream and device");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: out of host memory");
    b->ctx.assign(ctxs, ctxs + count);
    b->model = ctxs[0]->model;
    b->storage = ctxs[0]->storage;
    b->device = ctxs[0]->device;
    b->rho = ctxs[0]->rho[0] != nullptr;
    b->stream = ctxs[0]->stream;
    if (cudaMalloc(&b->d_lat, sizeof(BatchLattice) * count) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: cannot allocate descriptors");
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_config(lbm_batch* b, int block, int persistent) {
    if (!b) return LBM_EINVAL;
    if (block != 128 && block != 256) return bfail(b, LBM_EINVAL, "lbm_batch_set_config: block must be 128 or 256");
    if (block != b->block || (persistent != 0) != (b->persistent != 0)) drop_graph(b);
    b->block = block;
    b->persistent = persistent != 0;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, const int* steps) {
    if (!b) return LBM_EINVAL;
    if (!steps) return bfail(b, LBM_EINVAL, "lbm_batch_step: steps is NULL");
    const int count = (int)b->ctx.size();
    for (int k = 0; k < count; ++k)
        if (steps[k] < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: steps[%d] < 0", k);
    int dev = -1;
    BCUDA_TRY(b, cudaGetDevice(&dev));
    if (dev != b->device) BCUDA_TRY(b, cudaSetDevice(b->device));
    // A lattice whose planes fill the GPU runs its pairs of steps as two-step passes, launched as
    // lbm_step launches them (the same kernels, so the same results bit for bit); the others
    // advance together in the batched launches below. The passes are persistent launches over the
    // whole GPU, so a graph would save nothing on them.
    std::vector<int> batched(steps, steps + count);
    for (int k = 0; k < count; ++k) {
        lbm_ctx* c = b->ctx[k];
        if (steps[k] < 2 || pass_kind(c) == kPassNone) continue;
        const int64_t before = c->launches;
        const int rc = lbm_step(c, steps[k]);
        if (rc != LBM_OK) return bfail(b, rc, "lbm_batch_step: context %d: %s", k, c->err.c_str());
        b->launches += c->launches - before;
        batched[(size_t)k] = 0;
    }
    steps = batched.data();
    const BatchPlan p = plan_batch(b, steps);
    if (p.max_steps == 0) return LBM_OK;
    int rc;
    if ((rc = upload_tiles(b, p)) != LBM_OK) return rc;
    if ((rc = upload_batch(b, steps, p.max_steps)) != LBM_OK) return rc;
    // The sequence of launches depends only on the steps, the lattice sizes and the configuration;
    // everything else is read from the descriptors, so a captured graph replays for later calls.
    std::vector<long long> key{b->block, b->persistent};
    for (int k = 0; k < count; ++k) {
        key.push_back(steps[k]);
        key.push_back(b->ctx[k]->g.n);
        key.push_back(b->ctx[k]->n_special);
        key.push_back((long long)b->ctx[k]->sources.size());
    }
    int64_t launched = 0;
    if (b->stream == nullptr) {
        // The legacy default stream cannot be captured: launch directly.
        if ((rc = enqueue_steps(b, p, steps, &launched)) != LBM_OK) return rc;
    } else {
        if (!b->exec || key != b->graph_key) {
            drop_graph(b);
            cudaGraph_t graph = nullptr;
            BCUDA_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_steps(b, p, steps, &launched);
            cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
            if (rc != LBM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return bfail(b, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            b->graph_key = key;
        } else {
            for (int j = 0; j < p.max_steps; ++j)
                launched += (active_prefix(p, steps, j, p.tile_end) > 0) + (active_prefix(p, steps, j, p.stile_end) > 0);
        }
        BCUDA_TRY(b, cudaGraphLaunch(b->exec, b->stream));
    }
    b->launches += launched;
    for (int k = 0; k < count; ++k) {
        lbm_ctx* c = b->ctx[k];
        c->cur = (c->cur + steps[k]) & 1;
        c->t += steps[k];
    }
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* block_out, int* persistent_out) {
    if (!b) return LBM_EINVAL;
    if (trial_steps < 1) return bfail(b, LBM_EINVAL, "lbm_batch_autotune: trial_steps must be >= 1");
    const int count = (int)b->ctx.size();
    std::vector<int> ones((size_t)count, 1);
    cudaEvent_t e0, e1;
    BCUDA_TRY(b, cudaEventCreate(&e0));
    BCUDA_TRY(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_block = b->block, best_persistent = b->persistent;
    const int blocks[2] = {128, 256};
    int rc = LBM_OK;
    for (int bi = 0; bi < 2 && rc == LBM_OK; ++bi) {
        for (int pers = 0; pers < 2 && rc == LBM_OK; ++pers) {
            b->block = blocks[bi];
            b->persistent = pers;
            const BatchPlan p = plan_batch(b, ones.data());
            if ((rc = upload_tiles(b, p)) != LBM_OK) break;
            if ((rc = upload_batch(b, ones.data(), 1)) != LBM_OK) break;
            const BatchLaunch L = launch_config(b);
            const int nt = (int)p.tiles.size();
            // Step j = 0 repeatedly: reads the current buffers and rewrites the spare ones, so the
            // lattices' state is unchanged.
            auto run = [&]() {
                return b->model == LBM_MM ? mm_launch_batch_step(L, 0, nt, 0, b->stream)
                                          : hv_launch_batch_step(L, 0, nt, 0, b->stream);
            };
            run();
            cudaEventRecord(e0, b->stream);
            for (int s = 0; s < trial_steps; ++s) b->launches += run();
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                rc = bfail(b, LBM_ECUDA, "lbm_batch_autotune: trial launch failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_block = blocks[bi];
                best_persistent = pers;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graph(b);
    b->block = best_block;
    b->persistent = best_persistent;
    if (rc != LBM_OK) return rc;
    if (block_out) *block_out = best_block;
    if (persistent_out) *persistent_out = best_persistent;
    return LBM_OK;
}

int64_t lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : -1; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graph(b);
    if (b->d_lat) cudaFree(b->d_lat);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_stiles) cudaFree(b->d_stiles);
    if (b->d_stable) cudaFree(b->d_stable);
    delete b;
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// lbm_adjoint: loss over the next T steps and its gradient with respect to eps_r and sigma.
// ------------------------------------------------------------------------------------------------
namespace {

// Carves 256-byte-aligned pieces out of one allocation, in a fixed order.
struct Arena {
    size_t used = 0;
    char* base = nullptr;
    char* take(size_t bytes) {
        const size_t at = (used + 255) & ~(size_t)255;
        used = at + bytes;
        return base ? base + at : nullptr;
    }
};

int plane_size(const lbm_ctx* c, int axis) {
    return axis == 0 ? c->g.ny * c->g.nz : (axis == 1 ? c->g.nx * c->g.nz : c->g.nx * c->g.ny);
}

size_t record_bytes(const lbm_ctx* c) {
    return sizeof(float) * (size_t)c->g.n * (c->model == LBM_MM ? kRecordFloatsMM : kRecordFloatsHV);
}

// Work space of the adjoint: K record slots, n_ck checkpoint states (plus two scratch states to
// recompute through), two adjoint states, the gradient sums, the source-cell mask and the plane's
// loss slots. Returns its size; with a base, sets the pieces' addresses.
struct Layout {
    char *recs, *ck, *work, *nu, *mask, *loss;
    float *g_eps, *g_sig;
};
size_t adjoint_layout(const lbm_ctx* c, char* base, int K, int n_ck, int n_plane, Layout* L) {
    const size_t n = (size_t)c->g.n;
    const size_t state = (group_bytes(c->model, c->storage) + (c->model == LBM_HV ? pair_bytes(c->storage) : 0)) * n;
    Arena a;
    a.base = base;
    L->recs = a.take(record_bytes(c) * (size_t)K);
    L->ck = a.take(state * (size_t)n_ck);
    L->work = a.take(n_ck > 0 ? state * 2 : 0);
    L->nu = a.take(state * 2);
    L->g_eps = reinterpret_cast<float*>(a.take(sizeof(float) * n));
    L->g_sig = reinterpret_cast<float*>(a.take(sizeof(float) * n));
    L->mask = a.take(n);
    L->loss = a.take(sizeof(double) * ((size_t)n_plane + 3));
    return a.used;
}

// Segment length K (the final segment's records come from the forward pass) and the number of
// earlier segments, each recomputed once from a checkpoint.
struct AdjointPlan {
    int K, n_ck;
};
int earlier_segments(int steps, int K) { return K >= steps ? 0 : (steps - K + K - 1) / K; }

// Largest segment length whose work space fits in `budget` bytes (0 when none does).
int longest_fitting(const lbm_ctx* c, int steps, size_t budget) {
    Layout L;
    int best = 0;
    for (int K = 1; K <= steps; ++K)
        if (adjoint_layout(c, nullptr, K, earlier_segments(steps, K), 1, &L) <= budget) best = K;
    return best;
}

// The checkpointed mode's segment length for `steps` steps: the longest whose work space stays
// within that of segments of ceil(sqrt(steps)) steps (about sqrt(T) checkpoints and sqrt(T)
// records, the classic layout). Its memory grows like sqrt(T); the longer final segment, recorded
// by the forward pass, spares that many recomputed steps.
int sqrt_interval(const lbm_ctx* c, int steps) {
    const int k0 = std::min(steps, std::max(1, (int)std::ceil(std::sqrt((double)steps))));
    Layout L;
    const size_t classic = adjoint_layout(c, nullptr, k0, earlier_segments(steps, k0), 1, &L);
    return std::max(k0, longest_fitting(c, steps, classic));
}

// interval < 0: every record resident (K = steps); > 0: that segment length; 0: resident when its
// work space fits in half the free memory, else the sqrt(T) layout.
AdjointPlan adjoint_plan(const lbm_ctx* c, int steps, int interval) {
    int K = steps;
    if (interval > 0) {
        K = std::min(interval, steps);
    } else if (interval == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 0;
        }
        Layout L;
        const size_t avail = free_b + c->adj_ws_bytes;
        if (adjoint_layout(c, nullptr, steps, 0, 1, &L) > avail / 2) K = sqrt_interval(c, steps);
    }
    return AdjointPlan{K, earlier_segments(steps, K)};
}

}  // namespace

extern "C" int lbm_adjoint(lbm_ctx* ctx, int steps, int plane_axis, int plane_index, int checkpoint_interval,
                           double* loss_out, float* grad_eps_r, float* grad_sigma, int on_device) {
    if (!ctx) return LBM_EINVAL;
    if (steps < 1) return fail(ctx, LBM_EINVAL, "lbm_adjoint: steps must be >= 1");
    if (!loss_out) return fail(ctx, LBM_EINVAL, "lbm_adjoint: loss_out is NULL");
    if (ctx->storage != LBM_F32) return fail(ctx, LBM_EUNSUPPORTED, "lbm_adjoint: needs FP32 population storage");
    if (ctx->z_ghost) return fail(ctx, LBM_EUNSUPPORTED, "lbm_adjoint: not available on a z_ghost slab");
    const int dims[3] = {ctx->g.nx, ctx->g.ny, ctx->g.nz};
    if (plane_axis < 0 || plane_axis > 2 || plane_index < 0 || plane_index >= dims[plane_axis])
        return fail(ctx, LBM_EINVAL, "lbm_adjoint: plane (axis %d, index %d) outside the lattice", plane_axis,
                    plane_index);
    for (const HostSource& s : ctx->sources)
        for (int cell : s.cells) {
            const int x = cell % ctx->g.nx, y = (cell / ctx->g.nx) % ctx->g.ny, z = cell / (ctx->g.nx * ctx->g.ny);
            const int coord = plane_axis == 0 ? x : (plane_axis == 1 ? y : z);
            if (coord == plane_index)
                return fail(ctx, LBM_EINVAL, "lbm_adjoint: source cell %d lies in the loss plane", cell);
        }
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    const int n_plane = plane_size(ctx, plane_axis);
    // The T steps are cut into segments from the end: a final segment of K steps, whose records the
    // forward pass writes directly, and before it n_ck segments of K steps (the first one shorter)
    // whose starting states the forward pass keeps as checkpoints. Going backward, each earlier
    // segment is recomputed once from its checkpoint, writing its records into the same K slots.
    // K = steps keeps every record and recomputes nothing (the resident mode).
    const AdjointPlan plan = adjoint_plan(ctx, steps, checkpoint_interval);
    const bool resident = plan.K == steps;
    const int K = plan.K, n_ck = plan.n_ck;
    Layout Ly;
    const size_t need = adjoint_layout(ctx, nullptr, K, n_ck, n_plane, &Ly);
    if (need > ctx->adj_ws_bytes) {
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        free_dev(ctx->adj_ws);
        ctx->adj_ws_bytes = 0;
        if (cudaMalloc(&ctx->adj_ws, need) != cudaSuccess) {
            cudaGetLastError();
            ctx->adj_ws = nullptr;
            return fail(ctx, LBM_ENOMEM, "lbm_adjoint: cannot allocate %zu bytes of work space (%s, interval %d)",
                        need, resident ? "resident records" : "checkpoints", K);
        }
        ctx->adj_ws_bytes = need;
    }
    adjoint_layout(ctx, static_cast<char*>(ctx->adj_ws), K, n_ck, n_plane, &Ly);
    const int64_t n = ctx->g.n;
    const size_t b1 = group_bytes(ctx->model, ctx->storage) * (size_t)n;
    const size_t b2 = ctx->model == LBM_HV ? pair_bytes(ctx->storage) * (size_t)n : 0;
    const size_t state = b1 + b2;
    const size_t rec_bytes = record_bytes(ctx);
    CUDA_TRY(ctx, cudaMemsetAsync(Ly.g_eps, 0, sizeof(float) * (size_t)n, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(Ly.g_sig, 0, sizeof(float) * (size_t)n, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(Ly.mask, 0, (size_t)n, ctx->stream));
    if (ctx->n_special > 0) {
        std::vector<uint8_t> m((size_t)n, 0);
        for (const HostSource& s : ctx->sources)
            for (int cell : s.cells) m[(size_t)cell] = 1;
        CUDA_TRY(ctx, cudaMemcpyAsync(Ly.mask, m.data(), (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // m is released on return
    }
    auto state_ptrs = [&](char* base, void** p1, void** p2) {
        *p1 = base;
        *p2 = b2 ? base + b1 : nullptr;
    };
    // One forward step between explicit states, writing the adjoint record when rec is given. The
    // context's own pass also steps MM's tracked rest populations (it ends where lbm_step would).
    auto forward = [&](void* in1, void* in2, void* out1, void* out2, int64_t iter, bool own_state, void* rec) {
        StepArgs a = base_args(ctx);
        a.fin = in1;
        a.fin2 = in2;
        a.fout = out1;
        a.fout2 = out2;
        a.rho_in = own_state ? ctx->rho[ctx->cur] : nullptr;
        a.rho_out = own_state ? ctx->rho[1 - ctx->cur] : nullptr;
        a.rec = static_cast<float*>(rec);
        fill_scalars(ctx, a, iter);
        if (rec)
            return ctx->model == LBM_MM ? mm_launch_record_step(a, ctx->stream) : hv_launch_record_step(a, ctx->stream);
        return ctx->model == LBM_MM ? mm_launch_step(a, ctx->stream) : hv_launch_step(a, ctx->stream);
    };
    // Pairs of recording steps as one MM tiled pass wherever lbm_step would take that pass (the same
    // arithmetic: the same states and records, bit for bit).
    const bool tiled_rec = ctx->model == LBM_MM && pass_kind(ctx) == kPassTiled;
    const bool tiled_back = ctx->model == LBM_MM && ctx->fusion == 3 && pass_kind(ctx) == kPassTiled;
    if ((tiled_rec || tiled_back) && (rc = ensure_tiled(ctx)) != LBM_OK) return rc;
    TileArgs TA{};
    if (tiled_rec || tiled_back) {
        TA.tiles_x = tiled_tiles_x(ctx);
        TA.tiles_y = tiled_tiles_y(ctx);
        TA.chunk = tiled_chunk(ctx);
        TA.entry_off = ctx->d_tiled_off;
        TA.entries = ctx->d_tiled_entries;
    }
    // Two recording steps (iterations iter, iter + 1) from in1 to out1 as one tiled pass.
    auto forward2 = [&](void* in1, void* out1, int64_t iter, void* rec0, void* rec1) {
        StepArgs aA = base_args(ctx), aB = base_args(ctx);
        aA.fin = aB.fin = in1;
        aA.fout = aB.fout = out1;
        aA.rec = static_cast<float*>(rec0);
        aB.rec = static_cast<float*>(rec1);
        fill_scalars(ctx, aA, iter);
        fill_scalars(ctx, aB, iter + 1);
        return mm_launch_record_tile2(aA, aB, TA, ctx->stream);
    };
    int64_t launched = 0;
    const int64_t t0 = ctx->t;
    const int final_first = steps - K;  // first step of the final segment
    // first step of earlier segment k (0 .. n_ck - 1); segment k ends where k + 1 starts
    auto seg_first = [&](int k) { return std::max(0, final_first - (n_ck - k) * K); };
    // Forward pass: the state at the start of every earlier segment is kept, and the segment is
    // stepped as lbm_step steps it (two-step passes where they apply: the same bits as single
    // steps); the final segment is stepped writing its records, in pairs as recording tiled passes
    // where lbm_step takes the MM tiled pass, otherwise one step per launch.
    for (int k = 0; k < n_ck; ++k) {
        const int len = (k + 1 < n_ck ? seg_first(k + 1) : final_first) - seg_first(k);
        char* slot = Ly.ck + state * (size_t)k;
        CUDA_TRY(ctx, cudaMemcpyAsync(slot, ctx->buf[ctx->cur], b1, cudaMemcpyDeviceToDevice, ctx->stream));
        if (b2) CUDA_TRY(ctx, cudaMemcpyAsync(slot + b1, ctx->buf2[ctx->cur], b2, cudaMemcpyDeviceToDevice, ctx->stream));
        if ((rc = lbm_step(ctx, len)) != LBM_OK) return rc;
    }
    for (int s = final_first; s < steps; ++s) {
        char* rec = Ly.recs + rec_bytes * (size_t)(s - final_first);
        if (tiled_rec && s + 1 < steps) {
            launched += forward2(ctx->buf[ctx->cur], ctx->buf[1 - ctx->cur], t0 + s + 1, rec, rec + rec_bytes);
            ctx->t += 2;
            ++s;
        } else {
            launched += forward(ctx->buf[ctx->cur], ctx->buf2[ctx->cur], ctx->buf[1 - ctx->cur], ctx->buf2[1 - ctx->cur],
                                t0 + s + 1, true, rec);
            ctx->t += 1;
        }
        ctx->cur = 1 - ctx->cur;
    }
    if ((rc = check_launch(ctx, (int)launched)) != LBM_OK) return rc;
    launched = 0;
    // Terminal adjoint: nu^T = dL_T / df^T on the plane, and |E(T)|^2, from the final state.
    double* loss_plane = reinterpret_cast<double*>(Ly.loss);
    double* loss_dev = loss_plane + n_plane;
    int nu_cur = 0;
    CUDA_TRY(ctx, cudaMemsetAsync(Ly.nu, 0, state, ctx->stream));
    AdjointArgs A;
    memset(&A, 0, sizeof(A));
    A.grad_eps = Ly.g_eps;
    A.grad_sigma = grad_sigma ? Ly.g_sig : nullptr;  // not asked for: its sums are skipped
    A.special_mask = reinterpret_cast<const uint8_t*>(Ly.mask);
    A.plane_axis = plane_axis;
    A.plane_index = plane_index;
    A.loss_plane = loss_plane;
    A.a = base_args(ctx);
    A.a.fin = ctx->buf[ctx->cur];
    A.a.fin2 = ctx->buf2[ctx->cur];
    fill_scalars(ctx, A.a, t0 + steps + 1);
    state_ptrs(Ly.nu, &A.nu_out, &A.nu_out2);
    A.loss_active = 1;
    launched += ctx->model == LBM_MM ? mm_launch_adjoint_terminal(A, n_plane, ctx->stream)
                                     : hv_launch_adjoint_terminal(A, n_plane, ctx->stream);
    // Backward through the segment of steps first .. first + len - 1, whose records are in slots
    // 0 .. len - 1. With fusion mode 3, pairs of MM backward steps run as tiled passes (same
    // arithmetic and order of the gradient sums: the same bits). It is not the default: on GB300
    // (128^3, per-cell eps_r) a tiled pair takes 296 us against 2 x 141 for single steps.
    auto step_args = [&](AdjointArgs& X, int first, int j) {  // the backward step of record slot j
        const int64_t nstep = first + j;  // reverses forward iteration nstep + 1
        X.a = base_args(ctx);
        X.a.rec = reinterpret_cast<float*>(Ly.recs + rec_bytes * (size_t)j);
        fill_scalars(ctx, X.a, t0 + nstep + 1);
        X.loss_active = nstep >= 1 ? 1 : 0;
    };
    auto backward = [&](int first, int len) {
        for (int j = len - 1; j >= 0; --j) {
            step_args(A, first, j);
            state_ptrs(Ly.nu + state * (size_t)nu_cur, const_cast<void**>(&A.nu_in), const_cast<void**>(&A.nu_in2));
            state_ptrs(Ly.nu + state * (size_t)(1 - nu_cur), &A.nu_out, &A.nu_out2);
            if (tiled_back && j >= 1) {
                AdjointArgs A2 = A;  // the step of slot j - 1 writes nu_out; A reads nu_in
                step_args(A2, first, j - 1);
                launched += mm_launch_adjoint2(A, A2, TA, ctx->stream);
                --j;
            } else {
                launched += ctx->model == LBM_MM ? mm_launch_adjoint(A, ctx->stream) : hv_launch_adjoint(A, ctx->stream);
            }
            nu_cur = 1 - nu_cur;
        }
    };
    backward(final_first, K);
    for (int k = n_ck - 1; k >= 0; --k) {
        const int first = seg_first(k), len = (k + 1 < n_ck ? seg_first(k + 1) : final_first) - first;
        // Recompute the segment from its checkpoint through two scratch states, recording each step.
        void *i1, *i2, *o1, *o2;
        state_ptrs(Ly.ck + state * (size_t)k, &i1, &i2);
        int w = 0;  // the scratch state written next
        for (int j = 0; j < len; ++j) {
            state_ptrs(Ly.work + state * (size_t)w, &o1, &o2);
            char* rec = Ly.recs + rec_bytes * (size_t)j;
            if (tiled_rec && j + 1 < len) {
                launched += forward2(i1, o1, t0 + first + j + 1, rec, rec + rec_bytes);
                ++j;
            } else {
                launched += forward(i1, i2, o1, o2, t0 + first + j + 1, false, rec);
            }
            i1 = o1;
            i2 = o2;
            w ^= 1;
        }
        backward(first, len);
    }
    launched += launch_sum_doubles(loss_plane, n_plane, loss_dev, ctx->stream);
    if ((rc = check_launch(ctx, (int)launched)) != LBM_OK) return rc;
    CUDA_TRY(ctx, cudaMemcpyAsync(loss_out, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (grad_eps_r)
        CUDA_TRY(ctx, cudaMemcpyAsync(grad_eps_r, Ly.g_eps, sizeof(float) * n,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (grad_sigma)
        CUDA_TRY(ctx, cudaMemcpyAsync(grad_sigma, Ly.g_sig, sizeof(float) * n,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" int lbm_adjoint_release(lbm_ctx* ctx) {
    if (!ctx) return LBM_EINVAL;
    int rc;
    if ((rc = ensure_device(ctx)) != LBM_OK) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    free_dev(ctx->adj_ws);
    ctx->adj_ws_bytes = 0;
    return LBM_OK;
}

extern "C" int64_t lbm_adjoint_workspace_bytes(const lbm_ctx* ctx) { return ctx ? (int64_t)ctx->adj_ws_bytes : -1; }

extern "C" int lbm_adjoint_sqrt_interval(const lbm_ctx* ctx, int steps) {
    if (!ctx || steps < 1) return LBM_EINVAL;
    return sqrt_interval(ctx, steps);
}

// ------------------------------------------------------------------------------------------------
// z-slab halo: pack, unpack and exchange of the populations that cross a z face.
// ------------------------------------------------------------------------------------------------
namespace {

// Device planes of one face's crossing directions: for each direction its group plane (and, for
// HV, its pair plane). plane_z selects the plane; dirs are the directions crossing the face.
struct FacePlanes {
    int count = 0;
    char* ptr[8];
    size_t bytes[8];
};

FacePlanes face_planes(lbm_ctx* c, int plane_z, int vz_sign) {
    FacePlanes f;
    const size_t nxy = (size_t)c->g.nx * c->g.ny;
    const size_t n = (size_t)c->g.n;
    const size_t g_elem = group_bytes(c->model, c->storage) / (c->model == LBM_MM ? 12 : 6);
    int dirs[4];
    const int nd = c->model == LBM_MM ? mm_halo_dirs(vz_sign, dirs) : hv_halo_dirs(vz_sign, dirs);
    char* g = static_cast<char*>(c->buf[c->cur]);
    for (int k = 0; k < nd; ++k) {
        f.ptr[f.count] = g + g_elem * ((size_t)dirs[k] * n + (size_t)plane_z * nxy);
        f.bytes[f.count++] = g_elem * nxy;
    }
    if (c->model == LBM_HV) {
        const size_t p_elem = pair_bytes(c->storage) / 6;
        char* p = static_cast<char*>(c->buf2[c->cur]);
        for (int k = 0; k < nd; ++k) {
            f.ptr[f.count] = p + p_elem * ((size_t)dirs[k] * n + (size_t)plane_z * nxy);
            f.bytes[f.count++] = p_elem * nxy;
        }
    }
    return f;
}

// Outgoing values of face 0 (plane 1, v_z = -1) or face 1 (plane nz - 2, v_z = +1).
FacePlanes outgoing(lbm_ctx* c, int face) { return face == 0 ? face_planes(c, 1, -1) : face_planes(c, c->g.nz - 2, +1); }
// Ghost planes written by face 0 (plane 0, v_z = +1) or face 1 (plane nz - 1, v_z = -1).
FacePlanes incoming(lbm_ctx* c, int face) { return face == 0 ? face_planes(c, 0, +1) : face_planes(c, c->g.nz - 1, -1); }

size_t face_bytes(const FacePlanes& f) {
    size_t b = 0;
    for (int k = 0; k < f.count; ++k) b += f.bytes[k];
    return b;
}

int check_slab(lbm_ctx* c, const char* who) {
    if (!c) return LBM_EINVAL;
    if (!c->z_ghost) return fail(c, LBM_EINVAL, "%s: the context is not a z_ghost slab", who);
    return ensure_device(c);
}

// Staging buffer for host-side pack/unpack (one face), allocated on first use.
int halo_staging(lbm_ctx* c, size_t bytes, char** out) {
    if (c->halo_stage_bytes < bytes) {
        free_dev(c->halo_stage);
        c->halo_stage_bytes = 0;
        if (cudaMalloc(&c->halo_stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->halo_stage = nullptr;
            return fail(c, LBM_ENOMEM, "halo: cannot allocate %zu bytes of staging", bytes);
        }
        c->halo_stage_bytes = bytes;
    }
    *out = static_cast<char*>(c->halo_stage);
    return LBM_OK;
}

}  // namespace

extern "C" int64_t lbm_halo_bytes(const lbm_ctx* ctx) {
    if (!ctx || !ctx->z_ghost) return LBM_EINVAL;
    return (int64_t)face_bytes(outgoing(const_cast<lbm_ctx*>(ctx), 1));
}

extern "C" int lbm_halo_pack(lbm_ctx* ctx, int face, void* dst, int on_device) {
    int rc;
    if ((rc = check_slab(ctx, "lbm_halo_pack")) != LBM_OK) return rc;
    if (face != 0 && face != 1) return fail(ctx, LBM_EINVAL, "lbm_halo_pack: face must be 0 or 1");
    if (!dst) return fail(ctx, LBM_EINVAL, "lbm_halo_pack: dst is NULL");
    const FacePlanes f = outgoing(ctx, face);
    const size_t total = face_bytes(f);
    char* d = static_cast<char*>(dst);
    if (!on_device && (rc = halo_staging(ctx, total, &d)) != LBM_OK) return rc;
    HaloCopy h;
    memset(&h, 0, sizeof(h));
    size_t off = 0;
    for (int k = 0; k < f.count; ++k) {
        h.c[h.count++] = HaloChunk{f.ptr[k], d + off, (long long)f.bytes[k]};
        off += f.bytes[k];
    }
    if ((rc = check_launch(ctx, launch_halo_copy(h, ctx->stream))) != LBM_OK) return rc;
    if (!on_device) {
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, d, total, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBM_OK;
}

extern "C" int lbm_halo_unpack(lbm_ctx* ctx, int face, const void* src, int on_device) {
    int rc;
    if ((rc = check_slab(ctx, "lbm_halo_unpack")) != LBM_OK) return rc;
    if (face != 0 && face != 1) return fail(ctx, LBM_EINVAL, "lbm_halo_unpack: face must be 0 or 1");
    if (!src) return fail(ctx, LBM_EINVAL, "lbm_halo_unpack: src is NULL");
    const FacePlanes f = incoming(ctx, face);
    const size_t total = face_bytes(f);
    const char* s = static_cast<const char*>(src);
    if (!on_device) {
        char* stage = nullptr;
        if ((rc = halo_staging(ctx, total, &stage)) != LBM_OK) return rc;
        CUDA_TRY(ctx, cudaMemcpyAsync(stage, src, total, cudaMemcpyHostToDevice, ctx->stream));
        s = stage;
    }
    HaloCopy h;
    memset(&h, 0, sizeof(h));
    size_t off = 0;
    for (int k = 0; k < f.count; ++k) {
        h.c[h.count++] = HaloChunk{s + off, f.ptr[k], (long long)f.bytes[k]};
        off += f.bytes[k];
    }
    if ((rc = check_launch(ctx, launch_halo_copy(h, ctx->stream))) != LBM_OK) return rc;
    if (!on_device) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the host source may be reused
    return LBM_OK;
}

extern "C" int lbm_halo_exchange(lbm_ctx* lower, lbm_ctx* upper) {
    int rc;
    if (!lower || !upper) return LBM_EINVAL;
    if ((rc = check_slab(lower, "lbm_halo_exchange")) != LBM_OK) return rc;
    if ((rc = check_slab(upper, "lbm_halo_exchange")) != LBM_OK) return rc;
    if (lower->model != upper->model || lower->storage != upper->storage || lower->g.nx != upper->g.nx ||
        lower->g.ny != upper->g.ny || lower->device != upper->device || lower->stream != upper->stream)
        return fail(lower, LBM_EINVAL,
                    "lbm_halo_exchange: slabs must share model, storage, nx, ny, device and stream");
    const FacePlanes up_src = outgoing(lower, 1), up_dst = incoming(upper, 0);
    const FacePlanes down_src = outgoing(upper, 0), down_dst = incoming(lower, 1);
    HaloCopy h;
    memset(&h, 0, sizeof(h));
    for (int k = 0; k < up_src.count; ++k) h.c[h.count++] = HaloChunk{up_src.ptr[k], up_dst.ptr[k], (long long)up_src.bytes[k]};
    for (int k = 0; k < down_src.count; ++k)
        h.c[h.count++] = HaloChunk{down_src.ptr[k], down_dst.ptr[k], (long long)down_src.bytes[k]};
    return check_launch(lower, launch_halo_copy(h, lower->stream));
}

// ------------------------------------------------------------------------------------------------
// lbm_tiled_layout_check: the tiled pass's geometry, checked on the host with the kernel's own
// tile_coord and tile_core.
// ------------------------------------------------------------------------------------------------
extern "C" int lbm_tiled_layout_check(int nx, int ny) {
    if (nx < kTileEX || ny < kTileEY || (long long)nx * ny > (1 << 22)) return LBM_EINVAL;
    const int tx = (nx + kTileTX - 1) / kTileTX, ty = (ny + kTileTY - 1) / kTileTY;
    std::vector<int> owner((size_t)nx * ny, 0);
    for (int by = 0; by < ty; ++by)
        for (int bx = 0; bx < tx; ++bx) {
            std::vector<char> seen((size_t)nx * ny, 0);
            for (int local = 0; local < kTileThreads; ++local) {
                const int ex = local % kTileEX, ey = local / kTileEX;
                const int x = tile_coord(bx, ex, kTileTX, nx), y = tile_coord(by, ey, kTileTY, ny);
                // 1. an extended tile's positions are distinct cells
                if (seen[(size_t)x + (size_t)nx * y]++) return 1;
                if (!tile_core(local, bx, by, nx, ny)) continue;
                owner[(size_t)x + (size_t)nx * y] += 1;
                // 2. a core position's neighbours lie in the extended tile and are the lattice
                //    neighbours (periodic)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int nex = ex + dx, ney = ey + dy;
                        if (nex < 0 || nex >= kTileEX || ney < 0 || ney >= kTileEY) return 2;
                        if (tile_coord(bx, nex, kTileTX, nx) != (x + dx + nx) % nx ||
                            tile_coord(by, ney, kTileTY, ny) != (y + dy + ny) % ny)
                            return 3;
                    }
            }
        }
    // 3. the cores cover every cell exactly once
    for (int k : owner)
        if (k != 1) return 4;
    return LBM_OK;
}

// ------------------------------------------------------------------------------------------------
// lbm_fused_schedule_check: the two-step pass's order and dependency rules, checked on the host
// with the same functions the kernel uses (fused_phase, tile_window).
// ------------------------------------------------------------------------------------------------
extern "C" int lbm_fused_schedule_check(int nx, int ny, int nz, int R, int L, int tile_cells) {
    if (nx < 1 || ny < 1 || nz < 3 || L < 2 || R < L + 1 || nz < L + 1 || tile_cells < 1) return LBM_EINVAL;
    const long long nxy_ll = (long long)nx * ny;
    if (nxy_ll > (1 << 22)) return LBM_EINVAL;
    const int nxy = (int)nxy_ll, tiles = (nxy + tile_cells - 1) / tile_cells;
    // 1. the order visits every phase once
    std::vector<int> posA((size_t)nz, -1), posB((size_t)nz, -1);
    for (int q = 0; q < 2 * nz; ++q) {
        int type, plane;
        fused_phase(q, nz, L, &type, &plane);
        if (plane < 0 || plane >= nz) return 1;
        int& slot = type == kPhaseA ? posA[(size_t)plane] : posB[(size_t)plane];
        if (slot != -1) return 2;
        slot = q;
    }
    for (int p = 0; p < nz; ++p)
        if (posA[(size_t)p] < 0 || posB[(size_t)p] < 0) return 3;
    // 2. every wait (the kernel's own rule, fused_waits_on) targets an earlier phase; B(p) covers
    //    the three planes it reads
    for (int type = kPhaseA; type <= kPhaseB; ++type)
        for (int p = 0; p < nz; ++p) {
            int wtype = 0, q[3];
            const int nq = fused_waits_on(type, p, nz, R, &wtype, q);
            const int me = type == kPhaseA ? posA[(size_t)p] : posB[(size_t)p];
            for (int k = 0; k < nq; ++k) {
                if (q[k] < 0 || q[k] >= nz) return 4;
                if ((wtype == kPhaseA ? posA[(size_t)q[k]] : posB[(size_t)q[k]]) >= me) return 4;
            }
            if (type == kPhaseB) {
                bool reads[3] = {false, false, false};
                for (int k = 0; k < nq; ++k)
                    for (int d = -1; d <= 1; ++d)
                        if (wtype == kPhaseA && q[k] == (p + d + nz) % nz) reads[d + 1] = true;
                if (!(reads[0] && reads[1] && reads[2])) return 5;
            }
        }
    // 3. ring slots: when planes a < b share a slot (both in 1 .. nz - 2, a = b - R m), every B
    //    phase that reads a is ordered before A(b) through the chain of waits
    std::vector<std::vector<char>> before((size_t)(2 * nz), std::vector<char>((size_t)(2 * nz), 0));
    auto id = [&](int type, int p) { return (size_t)(type * nz + p); };
    std::vector<std::pair<int, int>> order((size_t)(2 * nz));
    for (int q = 0; q < 2 * nz; ++q) fused_phase(q, nz, L, &order[(size_t)q].first, &order[(size_t)q].second);
    for (int qi = 0; qi < 2 * nz; ++qi) {  // closure of the waits, in order (waits point backwards)
        const int type = order[(size_t)qi].first, p = order[(size_t)qi].second;
        int wtype = 0, q[3];
        const int nq = fused_waits_on(type, p, nz, R, &wtype, q);
        std::vector<char>& mine = before[id(type, p)];
        for (int k = 0; k < nq; ++k) {
            mine[id(wtype, q[k])] = 1;
            const std::vector<char>& theirs = before[id(wtype, q[k])];
            for (size_t z = 0; z < theirs.size(); ++z) mine[z] |= theirs[z];
        }
    }
    for (int b = 1; b <= nz - 2; ++b)
        for (int a = b - R; a >= 1; a -= R)
            for (int d = -1; d <= 1; ++d)
                if (!before[id(kPhaseA, b)][id(kPhaseB, (a + d + nz) % nz)]) return 6;
    // 4. tile windows: every cell a tile's cells pull from (x +- 1, y +- 1, periodic) lies in a tile
    //    of the window, and the window relation is symmetric (needed by the slot reuse waits)
    std::vector<char> in_window((size_t)tiles);
    std::vector<std::vector<char>> win((size_t)tiles);
    for (int j = 0; j < tiles; ++j) {
        int first, count;
        tile_window(j, tiles, tile_cells, nx, nxy, &first, &count);
        if (count < 1 || count > tiles || first < 0 || first >= tiles) return 7;
        std::fill(in_window.begin(), in_window.end(), 0);
        for (int k = 0, t = first; k < count; ++k, t = (t + 1) % tiles) in_window[(size_t)t] = 1;
        win[(size_t)j] = in_window;
        const int c1 = std::min((j + 1) * tile_cells, nxy);
        for (int c = j * tile_cells; c < c1; ++c) {
            const int x = c % nx, y = c / nx;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int cc = (x + dx + nx) % nx + nx * ((y + dy + ny) % ny);
                    if (!in_window[(size_t)(cc / tile_cells)]) return 8;
                }
        }
    }
    for (int a = 0; a < tiles; ++a)
        for (int b = 0; b < tiles; ++b)
            if (win[(size_t)a][(size_t)b] != win[(size_t)b][(size_t)a]) return 9;
    return LBM_OK;
}
