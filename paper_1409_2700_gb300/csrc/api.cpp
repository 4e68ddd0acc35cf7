// api.cpp -- the C ABI of libmcpt (declared in include/mcpt.h).
//
// Host-side runtime: argument validation, the monomer coefficient pool, a
// device arena for the integral blocks the library owns, the per-run dimer
// descriptors, wave planning under the scratch cap, kernel launches on the
// handle's stream, per-phase CUDA-event timing and the result copies.
#include "mcpt.h"
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <set>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

using namespace mcpt;

namespace {

thread_local std::string g_create_error;

struct MonomerRec {
    int nao, nocc;
    int offC, offE;
};

struct DfRec {                // a dimer of the density-fitted route
    int X, Y;
    const double* B;          // naux x (nX+nY)^2 FP64 on the device (library copy or borrowed)
    int naux;
    double s;
};

struct DimerRec {
    int X, Y;
    const double* E[2];
    long long st[2][3];
    bool computed;
    double* owned;        // library storage of host-given integrals (nullptr: never had any)
};

// Events of the timed runs since the last mcpt_collect_stats: per run
// [start, (first-half end, finish end) per wave, reduction end].
struct RunEvents {
    std::vector<cudaEvent_t> pool;
    std::vector<std::vector<cudaEvent_t>> pending;
    int runs = 0, launches = 0;
};

}  // namespace

struct mcpt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mcpt_precision prec = MCPT_FP64;
    int validate = 1;
    size_t wave_bytes = (size_t)1 << 30;
    std::string tune_cache;
    bool tune_loaded = false;
    std::map<std::string, TcTune> tuned;   // launch choices by wave signature
    int timing = 0;
    int graphs = 1;
    int coupling = 0;
    unsigned long long wait_ns = 0;  // limit of each device-side wait (0 = the kernels' default)
    int withhold = 0;                // test aid: see mcpt_options.withhold_load
    bool fp64_epilogue = false;      // mixed forms' energy epilogue on the FP64 pipe
    size_t mem_cap = 0;
    size_t mem_used = 0;

    std::vector<MonomerRec> mons;
    std::vector<std::vector<double>> monG, monU;   // Eq. (td2) monomer matrices (empty: zero)
    std::vector<DfRec> dfs;          // density-fitted route: dimers, scratch, results
    std::set<std::pair<int, int>> df_pairs;
    void* dDf = nullptr;
    size_t capDf = 0;
    double* dDfOut = nullptr;        // E2 (2 per dimer), monomer halves (2 N), totals (2)
    size_t capDfOut = 0;
    int* dDfLists = nullptr;
    size_t capDfLists = 0;
    bool df_ran = false;
    void* dTd2 = nullptr;            // Eq. (td2): batch arena, tables, monomer matrices, outputs
    size_t capTd2 = 0;
    void* dTd2Tab = nullptr;
    size_t capTd2Tab = 0;
    void* dTd2Mon = nullptr;
    size_t capTd2Mon = 0;
    void* dTd2Out = nullptr;
    size_t capTd2Out = 0;
    std::vector<double> hC, hE;
    double* dC = nullptr;
    float* dCf = nullptr;            // FP32 copy of the coefficient pool (mixed forms)
    double* dE = nullptr;
    size_t capC = 0, capCf = 0, capE = 0;
    bool mon_dirty = true;

    std::vector<DimerRec> dims;
    std::set<std::pair<int, int>> pairs;
    std::vector<void*> owned;        // arena chunks
    char* arena_ptr = nullptr;
    size_t arena_left = 0;

    void* dH = nullptr;              // first-half result of one wave (shared by every plan)
    size_t capH = 0;
    void* dVT = nullptr;             // coupling: every dimer's (ia|jb) and T = vD
    size_t capVT = 0;
    void* dCoup = nullptr;           // coupling tables: tiles, per-dimer info, monomer sizes, R offsets
    size_t capCoup = 0;
    double* dR = nullptr;            // coupling matrices R_X, per monomer
    size_t capR = 0;
    double* dPack[2] = {nullptr, nullptr};   // staging of host symmetry-packed integrals (two,
    size_t capPack[2] = {0, 0};              // filled alternately, each on its own copy stream,
    int pack_next = 0;                       // so that two host -> device copies run at once)
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    double* dS1 = nullptr;           // singles term: amplitudes t, the result s, per-dimer parts
    size_t capS1 = 0;
    long long s_total = 0;           // sum over monomers of o v
    long long s_parts = 0;           // sum over dimers of o_X v_X + o_Y v_Y
    std::vector<long long> r_off;    // host copy of the R offsets
    bool coupled = false;            // R holds the coupling of the current integrals
    double* dE2 = nullptr;
    size_t capE2 = 0;
    double* dMon = nullptr;
    size_t capMon = 0;
    int* dLists = nullptr;
    size_t capLists = 0;
    bool lists_dirty = true;
    double* dTot = nullptr;
    int* dFlag = nullptr;            // [0] validation flag, [1] device wait status

    struct Wave {
        int b, nd, max_rows, max_occ, max_ao;
        TcLaunch tc;
        size_t fin_off;              // byte offset of the wave's tasks in dFin
        int ntasks;                  // 0: one CTA per dimer (<= 32 AO)
        size_t part_off;             // first partial (pairs of doubles) in dPart
        int fin_warps;               // warps per CTA of the 32-AO second half
    };
    // A plan is the host work of a run that does not change between runs of
    // the same dimer range and precision (descriptors, waves, tensor maps and
    // work items, second-half tasks, the captured graph), with the device
    // buffers only it uses.  The context keeps several, so that runs that
    // alternate between ranges (waves of a streamed lattice) replan nothing.
    // A plan also names buffers every plan shares (dH, dE2, dMon, dLists, the
    // coefficient pools, the coupling arrays); when one of those is
    // reallocated `epoch` advances and plans built before it are rebuilt.
    struct Plan {
        bool valid = false;
        unsigned long long epoch = 0;      // the context's buffer epoch the plan was built against
        unsigned long long last_use = 0;
        mcpt_precision prec = MCPT_FP64;
        int first = 0, count = 0;
        std::vector<DimerDesc> hDesc;
        DimerDesc* dDesc = nullptr;
        size_t capDesc = 0;
        void* dWork = nullptr;             // tensor maps and work items of the tensor-core waves
        size_t capWork = 0;
        int* dFold = nullptr;              // split dimers: (dimer, first block slot, blocks)
        size_t capFold = 0;
        void* dFin = nullptr;              // second-half tasks of waves above 32 AO (+ first-task indices)
        size_t capFin = 0;
        double* dPart = nullptr;           // their FP64 partial sums
        size_t capPart = 0;
        std::vector<Wave> waves;
        double alg_bytes = 0, alg_flops = 0, alg_flops_half = 0;
        int nfold = 0;                     // split dimers whose block results are folded
        bool coupling = false;             // the plan stores (ia|jb), T and forms R
        int ntile[3] = {0, 0, 0};          // coupling output tiles of edge 64, 48, 32
        size_t off_tiles = 0, off_dims = 0, off_mdim = 0, off_roff = 0;   // into dCoup
        int nstiles = 0;                   // singles tiles
        size_t off_stiles = 0, off_soff = 0, off_poff = 0;
        cudaGraphExec_t graph = nullptr;   // the plan's launch sequence, captured on first use
        int graph_launches = 0;
    };
    std::vector<std::unique_ptr<Plan>> plans;
    Plan* coup = nullptr;                  // the plan whose run formed the current coupling
    unsigned long long epoch = 1, use_clock = 0;
    RunEvents rev;
    mcpt_run_stats stats{};
    bool ran = false;
    std::string err;
};

namespace {

mcpt_status fail(mcpt_ctx* h, mcpt_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(h, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(h, e_ == cudaErrorMemoryAllocation ? MCPT_ENOMEM : MCPT_ECUDA,           \
                        "CUDA error %s (%s) in %s", cudaGetErrorName(e_), cudaGetErrorString(e_), \
                        #call);                                                                  \
    } while (0)

mcpt_status dev_alloc(mcpt_ctx* h, void** p, size_t bytes)
{
    if (h->mem_cap && h->mem_used + bytes > h->mem_cap)
        return fail(h, MCPT_ENOMEM, "device memory cap of %zu bytes reached (%zu in use, %zu requested)",
                    h->mem_cap, h->mem_used, bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, MCPT_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    h->mem_used += bytes;
    return MCPT_OK;
}

void dev_free(mcpt_ctx* h, void* p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        h->mem_used -= bytes;
    }
}

// Grow-only device buffer.
template <typename T>
mcpt_status ensure(mcpt_ctx* h, T** p, size_t* cap, size_t bytes)
{
    if (*cap >= bytes && *p) return MCPT_OK;
    dev_free(h, *p, *cap);
    *p = nullptr;
    *cap = 0;
    void* q = nullptr;
    mcpt_status st = dev_alloc(h, &q, bytes);
    if (st) return st;
    *p = static_cast<T*>(q);
    *cap = bytes;
    return MCPT_OK;
}

// The two copy streams of the packed-integral staging buffers and their
// events, created on first use.
mcpt_status ensure_copy_streams(mcpt_ctx* h)
{
    for (int b = 0; b < 2; b++) {
        if (h->copy_stream[b]) continue;
        CK(h, cudaStreamCreateWithFlags(&h->copy_stream[b], cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming));
    }
    return MCPT_OK;
}

// A grow-only buffer that plans name: reallocating it advances the epoch, so
// the plans (and graphs) built against the old address are rebuilt.
template <typename T>
mcpt_status ensure_shared(mcpt_ctx* h, T** p, size_t* cap, size_t bytes)
{
    if (*cap >= bytes && *p) return MCPT_OK;
    h->epoch++;
    return ensure(h, p, cap, bytes);
}

void free_plan(mcpt_ctx* h, mcpt_ctx::Plan* P)
{
    if (P->graph) cudaGraphExecDestroy(P->graph);
    dev_free(h, P->dDesc, P->capDesc);
    dev_free(h, P->dWork, P->capWork);
    dev_free(h, P->dFold, P->capFold);
    dev_free(h, P->dFin, P->capFin);
    dev_free(h, P->dPart, P->capPart);
    *P = mcpt_ctx::Plan{};
}

// Forget every plan (the dimer or monomer set changed, or integral addresses
// did): their descriptors, slots and tensor maps no longer hold.
void drop_plans(mcpt_ctx* h)
{
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& P : h->plans) free_plan(h, P.get());
    h->plans.clear();
    h->coup = nullptr;
}

// Bump allocation from 256-byte aligned arena chunks (integral blocks owned
// by the library live here until mcpt_destroy).
mcpt_status arena_alloc(mcpt_ctx* h, size_t bytes, void** out)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes > h->arena_left) {
        size_t chunk = std::max(bytes, (size_t)512 << 20);
        void* p = nullptr;
        mcpt_status st = dev_alloc(h, &p, chunk);
        if (st) {
            if (chunk == bytes) return st;
            h->err.clear();
            st = dev_alloc(h, &p, bytes);   // retry with the exact size
            if (st) return st;
            chunk = bytes;
        }
        h->owned.push_back(p);
        h->arena_ptr = static_cast<char*>(p);
        h->arena_left = chunk;
    }
    *out = h->arena_ptr;
    h->arena_ptr += bytes;
    h->arena_left -= bytes;
    return MCPT_OK;
}

bool all_finite(const double* x, size_t n)
{
    for (size_t k = 0; k < n; k++)
        if (!std::isfinite(x[k])) return false;
    return true;
}

bool is_tensor_form(mcpt_precision p)
{
    return p == MCPT_TF32 || p == MCPT_BF16X3 || p == MCPT_BF16X2 || p == MCPT_FP64E;
}

TcKind tc_kind_of(mcpt_precision p)
{
    return p == MCPT_TF32 ? TC_TF32 : p == MCPT_BF16X2 ? TC_BF16X2 : p == MCPT_FP64E ? TC_FP64E : TC_BF16X3;
}

// Forms whose first-half result, second half, energy epilogue and stored
// coupling amplitudes are FP64 (the FP64 form and its tensor-core emulation).
bool fp64_data(mcpt_precision p) { return p == MCPT_FP64 || p == MCPT_FP64E; }

// Occupied pairs padded to 16 (N of the Kronecker tensor-core GEMM).
int npad_for(int oX, int oY) { return (oX * oY + 15) / 16 * 16; }

// Bytes of the first-half result of one dimer (both forms, pair-major).
size_t hbytes_for(mcpt_precision p, int nX, int nY, int oX, int oY)
{
    const size_t elem = fp64_data(p) ? sizeof(double) : sizeof(float);
    return 2 * (size_t)nX * nY * oX * oY * elem;
}

mcpt_status check_supported(mcpt_ctx* h, int d, int nX, int nY)
{
    switch (h->prec) {
    case MCPT_FP64:
        if (nX > 96 || nY > 96)
            return fail(h, MCPT_EUNSUPPORTED, "dimer %d: the FP64 form handles monomers of up to 96 AO", d);
        return MCPT_OK;
    case MCPT_FP32C:
        return MCPT_OK;
    case MCPT_TF32:
    case MCPT_BF16X3:
    case MCPT_BF16X2:
    case MCPT_FP64E:
        if ((nX & 1) || (nY & 1) || nX > kMaxAOTensor || nY > kMaxAOTensor)
            return fail(h, MCPT_EUNSUPPORTED,
                        "dimer %d: tensor-core forms need even AO counts <= %d (got %d, %d)", d,
                        kMaxAOTensor, nX, nY);
        return MCPT_OK;
    }
    return fail(h, MCPT_EINVAL, "unknown precision");
}

}  // namespace

void mcpt::set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }

// =================================================================== C ABI
extern "C" {

void mcpt_default_options(mcpt_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->device = 0;
    o->stream = nullptr;
    o->precision = MCPT_FP64;
    o->validate = 1;
    o->wave_bytes = (size_t)1 << 30;
    o->tune_cache = nullptr;
    o->timing = 0;
    o->mem_cap_bytes = 0;
    o->graphs = 1;
    o->coupling = 0;
}

mcpt_status mcpt_create(mcpt_handle* out, const mcpt_options* opt)
{
    if (!out) return fail(nullptr, MCPT_EINVAL, "mcpt_create: out is NULL");
    *out = nullptr;
    mcpt_options o;
    mcpt_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < MCPT_FP64 || o.precision > MCPT_FP64E)
        return fail(nullptr, MCPT_EINVAL, "mcpt_create: bad precision %d", (int)o.precision);
    if (o.withhold_load < 0) return fail(nullptr, MCPT_EINVAL, "mcpt_create: withhold_load %d < 0", o.withhold_load);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, MCPT_ECUDA, "mcpt_create: no CUDA device (%s)", cudaGetErrorString(e));
    }
    if (o.device < 0 || o.device >= ndev)
        return fail(nullptr, MCPT_EINVAL, "mcpt_create: device %d out of range (%d devices)", o.device, ndev);
    if ((e = cudaSetDevice(o.device)) != cudaSuccess)
        return fail(nullptr, MCPT_ECUDA, "mcpt_create: cudaSetDevice: %s", cudaGetErrorString(e));
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, o.device)) != cudaSuccess)
        return fail(nullptr, MCPT_ECUDA, "mcpt_create: %s", cudaGetErrorString(e));
    if (prop.major < 10)
        return fail(nullptr, MCPT_EUNSUPPORTED, "mcpt_create: device %s (sm_%d%d) is not a Blackwell GPU",
                    prop.name, prop.major, prop.minor);

    mcpt_ctx* h = new (std::nothrow) mcpt_ctx;
    if (!h) return fail(nullptr, MCPT_ENOMEM, "mcpt_create: out of host memory");
    h->device = o.device;
    h->prec = o.precision;
    h->validate = o.validate;
    h->wave_bytes = o.wave_bytes ? o.wave_bytes : ((size_t)1 << 30);
    h->tune_cache = o.tune_cache ? o.tune_cache : "";
    h->timing = o.timing;
    h->graphs = o.graphs;
    h->coupling = o.coupling;
    h->wait_ns = o.wait_limit_ns;
    h->withhold = o.withhold_load;
    h->fp64_epilogue = o.fp64_epilogue != 0;
    h->mem_cap = o.mem_cap_bytes;
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            delete h;
            return fail(nullptr, MCPT_ECUDA, "mcpt_create: stream: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    void* flag = nullptr;
    if (dev_alloc(h, &flag, 4 * sizeof(int)) != MCPT_OK) {
        std::string m = h->err;
        mcpt_destroy(h);
        return fail(nullptr, MCPT_ENOMEM, "mcpt_create: %s", m.c_str());
    }
    h->dFlag = static_cast<int*>(flag);
    cudaMemsetAsync(h->dFlag, 0, 4 * sizeof(int), h->stream);
    *out = h;
    return MCPT_OK;
}

mcpt_status mcpt_add_monomer(mcpt_handle h, const double* C, const double* eps, int nao, int nocc, int* id_out)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_add_monomer: NULL handle");
    if (!C || !eps) return fail(h, MCPT_EINVAL, "mcpt_add_monomer: C and eps must not be NULL");
    if (nao < 2 || nao > kMaxAOTensor)
        return fail(h, MCPT_EINVAL, "mcpt_add_monomer: nao=%d outside [2, %d]", nao, kMaxAOTensor);
    if (nocc < 1 || nocc > nao - 1)
        return fail(h, MCPT_EINVAL, "mcpt_add_monomer: nocc=%d outside [1, nao-1=%d]", nocc, nao - 1);
    if (h->validate && (!all_finite(C, (size_t)nao * nao) || !all_finite(eps, nao)))
        return fail(h, MCPT_EINVAL, "mcpt_add_monomer: non-finite value in C or eps");
    MonomerRec m{nao, nocc, (int)h->hC.size(), (int)h->hE.size()};
    h->hC.insert(h->hC.end(), C, C + (size_t)nao * nao);
    h->hE.insert(h->hE.end(), eps, eps + nao);
    h->mons.push_back(m);
    h->mon_dirty = true;
    drop_plans(h);
    h->lists_dirty = true;
    if (id_out) *id_out = (int)h->mons.size() - 1;
    return MCPT_OK;
}

static mcpt_status check_device_ptr(mcpt_handle h, const void* p, const char* who)
{
    cudaPointerAttributes pa;
    cudaError_t e = cudaPointerGetAttributes(&pa, p);
    if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != h->device) {
        cudaGetLastError();
        return fail(h, MCPT_EINVAL, "%s: on_device=1 but ao_eri is not device memory of device %d", who, h->device);
    }
    return MCPT_OK;
}

// Symmetry-packed integrals (X < Y): host data staged on the device, then
// expanded into `storage` (or new arena memory) in the BLOCKS layout; the
// record owns that storage.  Host data goes through two staging buffers
// filled on a copy stream, so that the copy of the next dimer overlaps the
// expansion of this one on the handle's stream.  Unless `async`, waits so
// that the caller's buffer is free on return.
static mcpt_status make_record_packed(mcpt_handle h, int X, int Y, const double* ao, int on_device,
                                      double* storage, bool async, DimerRec& r, const char* who)
{
    if (X > Y) return fail(h, MCPT_EINVAL, "%s: packed integrals must be given with X < Y", who);
    const int nX = h->mons[X].nao, nY = h->mons[Y].nao;
    const size_t blk = (size_t)nX * nX * nY * nY;
    const size_t np = packed_elems(nX, nY);
    mcpt_status st;
    const double* src = ao;
    int sb = -1;                         // staging buffer of host data
    if (on_device) {
        if ((st = check_device_ptr(h, ao, who))) return st;
        if (h->validate) {
            CK(h, cudaMemsetAsync(h->dFlag, 0, sizeof(int), h->stream));
            CK(h, launch_check_finite(ao, (long long)np, h->dFlag, h->stream));
            int flag = 0;
            CK(h, cudaMemcpyAsync(&flag, h->dFlag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            if (flag) return fail(h, MCPT_EINVAL, "%s: non-finite integral", who);
        }
    } else {
        if (h->validate && !all_finite(ao, np)) return fail(h, MCPT_EINVAL, "%s: non-finite integral", who);
        if ((st = ensure_copy_streams(h))) return st;
        sb = h->pack_next;
        h->pack_next ^= 1;
        if ((st = ensure(h, &h->dPack[sb], &h->capPack[sb], np * sizeof(double)))) return st;
        CK(h, cudaStreamWaitEvent(h->copy_stream[sb], h->ev_free[sb], 0));    // its last expansion has read it
        CK(h, cudaMemcpyAsync(h->dPack[sb], ao, np * sizeof(double), cudaMemcpyHostToDevice, h->copy_stream[sb]));
        CK(h, cudaEventRecord(h->ev_copied[sb], h->copy_stream[sb]));
        CK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[sb], 0));
        src = h->dPack[sb];
    }
    void* dst = storage;
    if (!dst && (st = arena_alloc(h, 2 * blk * sizeof(double), &dst))) return st;
    CK(h, launch_unpack(src, static_cast<double*>(dst), nX, nY, h->stream));
    if (sb >= 0) CK(h, cudaEventRecord(h->ev_free[sb], h->stream));
    if (!async) CK(h, cudaStreamSynchronize(h->stream));
    const double* b = static_cast<const double*>(dst);
    r.owned = static_cast<double*>(dst);
    r.E[0] = b;
    r.st[0][0] = (long long)nX * nY * nY; r.st[0][1] = (long long)nY * nY; r.st[0][2] = nY;
    r.E[1] = b + blk;
    r.st[1][0] = (long long)nY * nY * nX; r.st[1][1] = (long long)nY * nX; r.st[1][2] = nX;
    return MCPT_OK;
}

// Point record r (monomers X, Y in the caller's order; r.X < r.Y) at the
// dimer's integrals: device data in place (borrowed), host data copied into
// `storage` (2 nX^2 nY^2 doubles of library memory) or into new arena memory.
static mcpt_status make_record(mcpt_handle h, int X, int Y, const double* ao, mcpt_ao_layout layout, int on_device,
                               double* storage, bool async, DimerRec& r, const char* who)
{
    if (layout == MCPT_AO_PACKED) return make_record_packed(h, X, Y, ao, on_device, storage, async, r, who);
    const int nX = h->mons[X].nao, nY = h->mons[Y].nao, n = nX + nY;
    const size_t blk = (size_t)nX * nX * nY * nY;
    if (on_device) {
        cudaPointerAttributes pa;
        cudaError_t e = cudaPointerGetAttributes(&pa, ao);
        if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != h->device) {
            cudaGetLastError();
            return fail(h, MCPT_EINVAL, "%s: on_device=1 but ao_eri is not device memory of device %d", who,
                        h->device);
        }
        const long long n1 = n, n2 = n1 * n, n3 = n2 * n;
        if (layout == MCPT_AO_FULL) {
            r.E[0] = ao + nX * n1 + nX;                     // G[mu][nu][nX+lam][nX+sig]
            r.st[0][0] = n3; r.st[0][1] = n2; r.st[0][2] = n1;
            r.E[1] = ao + nX * n2 + nX * n1;                // G[mu][nX+lam][nX+sig][nu]
            r.st[1][0] = n3; r.st[1][1] = n2; r.st[1][2] = n1;
        } else {
            r.E[0] = ao;
            r.st[0][0] = (long long)nX * nY * nY; r.st[0][1] = (long long)nY * nY; r.st[0][2] = nY;
            r.E[1] = ao + blk;
            r.st[1][0] = (long long)nY * nY * nX; r.st[1][1] = (long long)nY * nX; r.st[1][2] = nX;
        }
        if (h->validate) {
            CK(h, cudaMemsetAsync(h->dFlag, 0, sizeof(int), h->stream));
            int dA[4] = {nX, nX, nY, nY}, dK[4] = {nX, nY, nY, nX};
            CK(h, launch_check_finite4(r.E[0], dA, r.st[0], h->dFlag, h->stream));
            CK(h, launch_check_finite4(r.E[1], dK, r.st[1], h->dFlag, h->stream));
            int flag = 0;
            CK(h, cudaMemcpyAsync(&flag, h->dFlag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            if (flag) return fail(h, MCPT_EINVAL, "%s: non-finite integral", who);
        }
    } else {
        // Host integrals: keep only the two blocks the term reads.  With X > Y
        // the dimer is stored as (Y, X): Y's functions become the first ones.
        const bool swap = X > Y;
        const int fX = swap ? nY : nX, fY = swap ? nX : nY;   // stored (first, second) sizes
        std::vector<double> tmp;
        const double* src = ao;
        if (layout == MCPT_AO_FULL || swap) {
            tmp.resize(2 * blk);
            double* A = tmp.data();
            double* K = tmp.data() + blk;
            // index of stored-order AO p in the caller's order
            auto map = [&](int p) { return swap ? (p < fX ? nX + p : p - fX) : p; };
            if (layout == MCPT_AO_FULL) {
                auto G = [&](int p, int q, int r_, int s) {
                    return ao[(((size_t)map(p) * n + map(q)) * n + map(r_)) * n + map(s)];
                };
                for (int mu = 0; mu < fX; mu++)
                    for (int nu = 0; nu < fX; nu++)
                        for (int la = 0; la < fY; la++)
                            for (int sg = 0; sg < fY; sg++)
                                A[(((size_t)mu * fX + nu) * fY + la) * fY + sg] = G(mu, nu, fX + la, fX + sg);
                for (int mu = 0; mu < fX; mu++)
                    for (int la = 0; la < fY; la++)
                        for (int sg = 0; sg < fY; sg++)
                            for (int nu = 0; nu < fX; nu++)
                                K[(((size_t)mu * fY + la) * fY + sg) * fX + nu] = G(mu, fX + la, fX + sg, nu);
            } else {
                // caller's blocks are (X first): A0[nX][nX][nY][nY], K0[nX][nY][nY][nX];
                // with real-orbital integral symmetry (pq|rs) = (rs|pq) = (qp|sr):
                // (YY|XX) = A0 transposed, (YX|XY) = K0 with both pairs swapped.
                const double* A0 = ao;
                const double* K0 = ao + blk;
                for (int mu = 0; mu < fX; mu++)
                    for (int nu = 0; nu < fX; nu++)
                        for (int la = 0; la < fY; la++)
                            for (int sg = 0; sg < fY; sg++)
                                A[(((size_t)mu * fX + nu) * fY + la) * fY + sg] =
                                    A0[(((size_t)la * nX + sg) * nY + mu) * nY + nu];
                for (int mu = 0; mu < fX; mu++)
                    for (int la = 0; la < fY; la++)
                        for (int sg = 0; sg < fY; sg++)
                            for (int nu = 0; nu < fX; nu++)
                                K[(((size_t)mu * fY + la) * fY + sg) * fX + nu] =
                                    K0[(((size_t)la * nY + mu) * nY + nu) * nX + sg];
            }
            src = tmp.data();
        }
        if (h->validate && !all_finite(src, 2 * blk))
            return fail(h, MCPT_EINVAL, "%s: non-finite integral", who);
        void* dst = storage;
        if (!dst) {
            mcpt_status st = arena_alloc(h, 2 * blk * sizeof(double), &dst);
            if (st) return st;
        }
        CK(h, cudaMemcpyAsync(dst, src, 2 * blk * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        // the caller may free its buffer on return, unless it asked for an
        // asynchronous copy of its own (unrelabelled) blocks
        if (!(async && src == ao)) CK(h, cudaStreamSynchronize(h->stream));
        const double* b = static_cast<const double*>(dst);
        r.owned = static_cast<double*>(dst);
        r.E[0] = b;
        r.st[0][0] = (long long)fX * fY * fY; r.st[0][1] = (long long)fY * fY; r.st[0][2] = fY;
        r.E[1] = b + blk;
        r.st[1][0] = (long long)fY * fY * fX; r.st[1][1] = (long long)fY * fX; r.st[1][2] = fX;
    }
    return MCPT_OK;
}

mcpt_status mcpt_add_dimer(mcpt_handle h, int X, int Y, const double* ao, mcpt_ao_layout layout, int on_device,
                           int* id_out)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_add_dimer: NULL handle");
    const int N = (int)h->mons.size();
    if (X < 0 || X >= N || Y < 0 || Y >= N)
        return fail(h, MCPT_EINVAL, "mcpt_add_dimer: unknown monomer id (%d, %d) of %d", X, Y, N);
    if (X == Y) return fail(h, MCPT_EINVAL, "mcpt_add_dimer: X == Y == %d", X);
    if (!ao) return fail(h, MCPT_EINVAL, "mcpt_add_dimer: ao_eri is NULL");
    if (layout != MCPT_AO_FULL && layout != MCPT_AO_BLOCKS && layout != MCPT_AO_PACKED)
        return fail(h, MCPT_EINVAL, "mcpt_add_dimer: bad layout %d", (int)layout);
    if (on_device && X > Y)
        return fail(h, MCPT_EINVAL, "mcpt_add_dimer: device integrals must be given with X < Y");
    const std::pair<int, int> key(std::min(X, Y), std::max(X, Y));
    if (h->pairs.count(key)) return fail(h, MCPT_EINVAL, "mcpt_add_dimer: duplicate dimer (%d, %d)", X, Y);
    CK(h, cudaSetDevice(h->device));
    DimerRec r{};
    r.X = key.first;
    r.Y = key.second;
    r.computed = false;
    mcpt_status st = make_record(h, X, Y, ao, layout, on_device, nullptr, false, r, "mcpt_add_dimer");
    if (st) return st;
    h->dims.push_back(r);
    h->pairs.insert(key);
    h->coupled = false;
    drop_plans(h);
    h->lists_dirty = true;
    if (id_out) *id_out = (int)h->dims.size() - 1;
    return MCPT_OK;
}

mcpt_status mcpt_update_dimer(mcpt_handle h, int id, const double* ao, mcpt_ao_layout layout, int on_device,
                              int flags)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_update_dimer: NULL handle");
    if (id < 0 || id >= (int)h->dims.size())
        return fail(h, MCPT_EINVAL, "mcpt_update_dimer: unknown dimer id %d of %zu", id, h->dims.size());
    if (!ao) return fail(h, MCPT_EINVAL, "mcpt_update_dimer: ao_eri is NULL");
    if (layout != MCPT_AO_FULL && layout != MCPT_AO_BLOCKS && layout != MCPT_AO_PACKED)
        return fail(h, MCPT_EINVAL, "mcpt_update_dimer: bad layout %d", (int)layout);
    if (flags & ~MCPT_UPDATE_ASYNC) return fail(h, MCPT_EINVAL, "mcpt_update_dimer: unknown flags 0x%x", flags);
    CK(h, cudaSetDevice(h->device));
    const DimerRec& old = h->dims[id];
    DimerRec r = old;
    r.computed = false;
    // host data (and packed data from anywhere) reuses the dimer's library
    // storage when it has some
    const bool packed = layout == MCPT_AO_PACKED;
    mcpt_status st = make_record(h, old.X, old.Y, ao, layout, on_device, on_device && !packed ? nullptr : old.owned,
                                 (flags & MCPT_UPDATE_ASYNC) != 0, r, "mcpt_update_dimer");
    if (st) return st;
    if (on_device && !packed) r.owned = old.owned;     // keep the storage for a later host update
    if (r.E[0] != old.E[0] || r.E[1] != old.E[1] || std::memcmp(r.st, old.st, sizeof r.st))
        drop_plans(h);                      // the tensor maps name the old addresses
    h->dims[id] = r;
    h->coupled = false;
    return MCPT_OK;
}

// Many dimers' new integrals in one call (host memory).  Packed data of
// dimers that lie back to back in the caller's buffer is copied in chunks of
// up to kUpdateChunk bytes (at most kUnpackBatch dimers) through the two
// staging buffers on the copy stream, and each chunk is expanded into the
// dimers' storage by one launch on the handle's stream; BLOCKS data goes
// dimer by dimer straight into the storage (one copy each is already
// link-bound).
constexpr size_t kUpdateChunk = (size_t)256 << 20;

mcpt_status mcpt_update_dimers(mcpt_handle h, int first, int count, const double* ao, const size_t* offsets,
                               mcpt_ao_layout layout, int flags)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_update_dimers: NULL handle");
    const int D = (int)h->dims.size();
    if (first < 0 || count < 0 || first + count > D)
        return fail(h, MCPT_EINVAL, "mcpt_update_dimers: [%d, %d) outside [0, %d)", first, first + count, D);
    if (count == 0) return MCPT_OK;
    if (!ao || !offsets) return fail(h, MCPT_EINVAL, "mcpt_update_dimers: ao_eri or offsets is NULL");
    if (layout != MCPT_AO_BLOCKS && layout != MCPT_AO_PACKED)
        return fail(h, MCPT_EINVAL, "mcpt_update_dimers: layout must be MCPT_AO_BLOCKS or MCPT_AO_PACKED");
    if (flags & ~MCPT_UPDATE_ASYNC) return fail(h, MCPT_EINVAL, "mcpt_update_dimers: unknown flags 0x%x", flags);
    if (layout == MCPT_AO_BLOCKS) {
        for (int k = 0; k < count; k++) {
            mcpt_status st = mcpt_update_dimer(h, first + k, ao + offsets[k], layout, 0, flags);
            if (st) return st;
        }
        return MCPT_OK;
    }
    CK(h, cudaSetDevice(h->device));
    mcpt_status st;
    std::vector<size_t> np(count);
    bool moved = false;
    for (int k = 0; k < count; k++) {
        DimerRec& r = h->dims[first + k];
        const int nX = h->mons[r.X].nao, nY = h->mons[r.Y].nao;
        np[k] = packed_elems(nX, nY);
        if (h->validate && !all_finite(ao + offsets[k], np[k]))
            return fail(h, MCPT_EINVAL, "mcpt_update_dimers: non-finite integral (dimer %d)", first + k);
        const size_t blk = (size_t)nX * nX * nY * nY;
        if (!r.owned) {                       // only ever borrowed device data: storage of its own
            void* dst = nullptr;
            if ((st = arena_alloc(h, 2 * blk * sizeof(double), &dst))) return st;
            r.owned = static_cast<double*>(dst);
        }
        if (r.E[0] != r.owned) {              // the record points at borrowed data: back to the storage
            r.E[0] = r.owned;
            r.st[0][0] = (long long)nX * nY * nY; r.st[0][1] = (long long)nY * nY; r.st[0][2] = nY;
            r.E[1] = r.owned + blk;
            r.st[1][0] = (long long)nY * nY * nX; r.st[1][1] = (long long)nY * nX; r.st[1][2] = nX;
            moved = true;
        }
    }
    if (moved) drop_plans(h);                 // the tensor maps name the old addresses
    if ((st = ensure_copy_streams(h))) return st;
    const size_t chunk_elems = kUpdateChunk / sizeof(double);
    for (int k = 0; k < count;) {
        size_t elems = np[k];
        int k2 = k + 1;
        while (k2 < count && k2 - k < kUnpackBatch && offsets[k2] == offsets[k2 - 1] + np[k2 - 1] &&
               elems + np[k2] <= chunk_elems) {
            elems += np[k2];
            k2++;
        }
        const int sb = h->pack_next;
        h->pack_next ^= 1;
        if ((st = ensure(h, &h->dPack[sb], &h->capPack[sb], elems * sizeof(double)))) return st;
        CK(h, cudaStreamWaitEvent(h->copy_stream[sb], h->ev_free[sb], 0));    // its last expansion has read it
        CK(h, cudaMemcpyAsync(h->dPack[sb], ao + offsets[k], elems * sizeof(double), cudaMemcpyHostToDevice,
                              h->copy_stream[sb]));
        CK(h, cudaEventRecord(h->ev_copied[sb], h->copy_stream[sb]));
        CK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[sb], 0));
        UnpackBatch B;
        B.staging = h->dPack[sb];
        B.n = k2 - k;
        for (int j = 0; j < B.n; j++) {
            const DimerRec& r = h->dims[first + k + j];
            B.e[j] = UnpackEntry{(long long)(offsets[k + j] - offsets[k]), r.owned, h->mons[r.X].nao,
                                 h->mons[r.Y].nao};
        }
        CK(h, launch_unpack_batch(B, h->stream));
        CK(h, cudaEventRecord(h->ev_free[sb], h->stream));
        k = k2;
    }
    for (int k = 0; k < count; k++) h->dims[first + k].computed = false;
    h->coupled = false;
    if (!(flags & MCPT_UPDATE_ASYNC)) CK(h, cudaStreamSynchronize(h->stream));
    return MCPT_OK;
}

mcpt_status mcpt_set_precision(mcpt_handle h, mcpt_precision p)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_set_precision: NULL handle");
    if (p < MCPT_FP64 || p > MCPT_FP64E) return fail(h, MCPT_EINVAL, "mcpt_set_precision: bad precision %d", (int)p);
    h->prec = p;                            // plans are kept per precision
    return MCPT_OK;
}

static mcpt_status upload_static(mcpt_handle h)
{
    if (h->mon_dirty) {
        mcpt_status st = ensure_shared(h, &h->dC, &h->capC, h->hC.size() * sizeof(double));
        if (st) return st;
        st = ensure_shared(h, &h->dE, &h->capE, h->hE.size() * sizeof(double));
        if (st) return st;
        st = ensure_shared(h, &h->dCf, &h->capCf, h->hC.size() * sizeof(float));
        if (st) return st;
        std::vector<float> cf(h->hC.begin(), h->hC.end());
        CK(h, cudaMemcpyAsync(h->dC, h->hC.data(), h->hC.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->dCf, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->dE, h->hE.data(), h->hE.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->mon_dirty = false;
    }
    if (h->lists_dirty) {
        // CSR of dimers per monomer, ascending dimer id
        const int N = (int)h->mons.size(), D = (int)h->dims.size();
        std::vector<int> cnt(N + 1, 0), lists(N + 1 + 2 * (size_t)D);
        for (const auto& r : h->dims) { cnt[r.X + 1]++; cnt[r.Y + 1]++; }
        for (int m = 0; m < N; m++) cnt[m + 1] += cnt[m];
        std::copy(cnt.begin(), cnt.end(), lists.begin());
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int d = 0; d < D; d++) {
            lists[N + 1 + fill[h->dims[d].X]++] = d;
            lists[N + 1 + fill[h->dims[d].Y]++] = d;
        }
        mcpt_status st = ensure_shared(h, &h->dLists, &h->capLists, lists.size() * sizeof(int));
        if (st) return st;
        CK(h, cudaMemcpyAsync(h->dLists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->lists_dirty = false;
    }
    return MCPT_OK;
}

// Host work of a run that does not change between runs of the same dimer set:
// descriptors, wave split under the scratch cap, scratch buffers, and (for
// the tensor-core forms) tensor maps and ordered work items, all uploaded.
// ------------------------------------------------------------------ autotuner
// With options.tune_cache set, the launch choices of each tensor-core wave
// (kernel variant, staging depth, grid) are measured once per wave signature
// -- precision, device, and the multiset of dimer shapes (nX, nY, oX, oY) --
// and kept as one text line per signature in that file:
//   <key> <variant+1> <stages> <grid> <ms>
// Later plans with the same signature reuse the line without timing.
static std::string tune_key(mcpt_ctx* h, mcpt_precision prec, const DimerDesc* d, int nd)
{
    std::map<std::vector<int>, int> sig;
    for (int k = 0; k < nd; k++) sig[{d[k].nX, d[k].nY, d[k].oX, d[k].oY}]++;
    unsigned long long f = 1469598103934665603ull;        // FNV-1a over the signature
    auto mix = [&](long long v) {
        for (int b = 0; b < 8; b++) {
            f ^= (unsigned long long)((v >> (8 * b)) & 0xff);
            f *= 1099511628211ull;
        }
    };
    for (auto& kv : sig) {
        for (int v : kv.first) mix(v);
        mix(kv.second);
    }
    cudaDeviceProp prop;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) dev = prop.name;
    for (auto& c : dev)
        if (c == ' ') c = '_';
    char buf[160];
    snprintf(buf, sizeof buf, "%s:%s:%d:%016llx", prec == MCPT_TF32 ? "tf32" : prec == MCPT_BF16X2 ? "bf16x2" : prec == MCPT_FP64E ? "fp64e" : "bf16x3",
             dev.c_str(), nd, f);
    return buf;
}

static void tune_load(mcpt_ctx* h)
{
    if (h->tune_loaded) return;
    h->tune_loaded = true;
    std::ifstream in(h->tune_cache);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string key;
        TcTune t{};
        double ms = 0;
        if (ls >> key >> t.variant1 >> t.sf >> t.grid >> ms) h->tuned[key] = t;
    }
}

// Time every candidate launch of wave `wv` on the handle's stream (one
// warm-up launch, then three timed ones) and return the fastest.
static mcpt_status tune_wave(mcpt_handle h, const mcpt_ctx::Plan& P, TcKind kind, const mcpt_ctx::Wave& wv,
                             void* work, size_t work_bytes, TcTune* best, float* best_ms)
{
    TcTune cand[16];
    const int n = tc_candidates(kind, P.hDesc.data() + wv.b, wv.nd, cand, 16);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    *best_ms = 1e30f;
    *best = TcTune{};
    for (int c = 0; c < n; c++) {
        TcLaunch L{};
        char err[256] = {0};
        if (tc_prepare(kind, P.hDesc.data() + wv.b, P.dDesc + wv.b, wv.nd, h->dCf, h->dC, h->dH,
                       work, work_bytes, h->dFlag + 1, h->stream, &cand[c], &L, err, sizeof err) != cudaSuccess)
            continue;
        cudaError_t e = tc_launch(L, h->stream);
        e = e ? e : cudaEventRecord(e0, h->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; r++) e = tc_launch(L, h->stream);
        e = e ? e : cudaEventRecord(e1, h->stream);
        e = e ? e : cudaEventSynchronize(e1);
        float ms = 0;
        e = e ? e : cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(h, MCPT_ECUDA, "autotuner: %s", cudaGetErrorString(e));
        }
        if (ms < *best_ms) {
            *best_ms = ms;
            *best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(h, cudaMemsetAsync(h->dFlag + 1, 0, sizeof(int), h->stream));
    return MCPT_OK;
}

static mcpt_status build_plan(mcpt_handle h, mcpt_ctx::Plan& P, int first, int count)
{
    const int D = (int)h->dims.size();
    const int N = (int)h->mons.size();
    const mcpt_precision prec = h->prec;
    P.valid = false;
    P.waves.clear();
    if (P.graph) {
        cudaGraphExecDestroy(P.graph);
        P.graph = nullptr;
    }

    P.hDesc.clear();
    // the coupling needs every dimer's amplitudes at once: full runs only
    const bool coupled_plan = h->coupling && first == 0 && count == D;
    long long vt_total = 0;
    std::vector<std::pair<int, int>> waves;   // [begin, end) into hDesc
    std::vector<int> fold;                    // split dimers: (dimer, first block slot, blocks)
    int nblk_extra = 0;                       // result slots of blocks past the D dimers
    size_t wave_h = 0, max_wave_h = 0;
    int wbeg = 0;
    double alg_bytes = 0.0, alg_flops = 0.0, alg_flops_half = 0.0;
    for (int k = 0; k < count; k++) {
        const int d = first + k;
        const DimerRec& r = h->dims[d];
        const MonomerRec& mX = h->mons[r.X];
        const MonomerRec& mY = h->mons[r.Y];
        mcpt_status st = check_supported(h, d, mX.nao, mY.nao);
        if (st) return st;
        DimerDesc base{};
        base.E[0] = r.E[0];
        base.E[1] = r.E[1];
        std::memcpy(base.st, r.st, sizeof base.st);
        base.nX = mX.nao; base.nY = mY.nao;
        base.cXv = mX.offC + mX.nocc; base.cYv = mY.offC + mY.nocc;
        base.eXv = mX.offE + mX.nocc; base.eYv = mY.offE + mY.nocc;
        base.vX = mX.nao - mX.nocc; base.vY = mY.nao - mY.nocc;
        base.X = r.X; base.Y = r.Y;
        base.oXt = mX.nocc; base.oYt = mY.nocc;
        base.vt_off = -1;
        if (coupled_plan) {
            base.vt_off = vt_total;
            vt_total += 2LL * mX.nocc * (mX.nao - mX.nocc) * mY.nocc * (mY.nao - mY.nocc);
        }
        // tensor-core work items hold at most kMaxOccTensorX occupied orbitals of X
        // and kMaxOccTensor of Y: larger occupations run as near-equal blocks of (i, j)
        const int bx = is_tensor_form(prec) ? (mX.nocc + kMaxOccTensorX - 1) / kMaxOccTensorX : 1;
        const int by = is_tensor_form(prec) ? (mY.nocc + kMaxOccTensor - 1) / kMaxOccTensor : 1;
        if (bx * by > 1) {
            fold.insert(fold.end(), {d, D + nblk_extra, bx * by});
        }
        for (int ib = 0; ib < bx; ib++)
            for (int jb = 0; jb < by; jb++) {
                DimerDesc dd = base;
                const int i0 = ib * mX.nocc / bx, i1 = (ib + 1) * mX.nocc / bx;
                const int j0 = jb * mY.nocc / by, j1 = (jb + 1) * mY.nocc / by;
                dd.oX = i1 - i0; dd.oY = j1 - j0;
                dd.iX0 = i0; dd.jY0 = j0;
                dd.cX = mX.offC + i0; dd.cY = mY.offC + j0;
                dd.eX = mX.offE + i0; dd.eY = mY.offE + j0;
                dd.npad = npad_for(dd.oX, dd.oY);
                dd.slot = bx * by > 1 ? D + nblk_extra++ : d;
                const size_t hb = hbytes_for(prec, dd.nX, dd.nY, dd.oX, dd.oY);
                const size_t elem = fp64_data(prec) ? 8 : 4;
                const int kk = (int)P.hDesc.size();
                if (kk > wbeg && (wave_h + hb > h->wave_bytes || kk - wbeg >= 65535)) {
                    waves.emplace_back(wbeg, kk);
                    max_wave_h = std::max(max_wave_h, wave_h);
                    wbeg = kk;
                    wave_h = 0;
                }
                dd.h_off = (long long)(wave_h / elem);
                wave_h += hb;
                P.hDesc.push_back(dd);
            }
        const double nx = mX.nao, ny = mY.nao, ox = mX.nocc, oy = mY.nocc, vx = nx - ox, vy = ny - oy;
        alg_bytes += 2.0 * nx * nx * ny * ny * 8.0;
        alg_flops += 2.0 * 2.0 * (nx * nx * ny * ny * oy + ox * nx * nx * ny * oy + ox * nx * oy * ny * vy +
                                  ox * vx * oy * vy * nx);
        alg_flops_half += 2.0 * 2.0 * (nx * nx * ny * ny * oy + ox * nx * nx * ny * oy);
    }
    const int ndesc = (int)P.hDesc.size();
    waves.emplace_back(wbeg, ndesc);
    max_wave_h = std::max(max_wave_h, wave_h);

    mcpt_status st = upload_static(h);
    if (st) return st;
    if ((st = ensure(h, &P.dDesc, &P.capDesc, ndesc * sizeof(DimerDesc)))) return st;
    if ((st = ensure_shared(h, &h->dH, &h->capH, max_wave_h))) return st;
    if (!fold.empty() && (st = ensure(h, &P.dFold, &P.capFold, fold.size() * sizeof(int)))) return st;
    // per-dimer results, then the results of split dimers' blocks (kept across
    // plans: a larger array copies the dimers' results over)
    const size_t e2_bytes = (size_t)2 * (D + nblk_extra) * sizeof(double);
    if (h->capE2 < e2_bytes) {
        double* old = h->dE2;
        const size_t old_cap = h->capE2;
        void* q = nullptr;
        if ((st = dev_alloc(h, &q, e2_bytes))) return st;
        if (old) {
            CK(h, cudaMemcpyAsync(q, old, std::min(old_cap, (size_t)2 * D * sizeof(double)), cudaMemcpyDeviceToDevice,
                                  h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            dev_free(h, old, old_cap);
        }
        h->dE2 = static_cast<double*>(q);
        h->capE2 = e2_bytes;
        h->epoch++;
    }
    // monomer halves, totals, then the reduction's scratch
    if ((st = ensure_shared(h, &h->dMon, &h->capMon, ((size_t)2 * N + 2 + 4 * kReduceBlocks) * sizeof(double))))
        return st;
    h->dTot = h->dMon + 2 * N;
    std::vector<size_t> work_off;
    if (is_tensor_form(prec)) {
        size_t total = 0;
        for (auto& w : waves) {
            work_off.push_back(total);
            total += (tc_work_bytes(tc_kind_of(prec), P.hDesc.data() + w.first, w.second - w.first) + 255) & ~(size_t)255;
        }
        if ((st = ensure(h, &P.dWork, &P.capWork, total))) return st;
    }
    P.coupling = coupled_plan;
    P.ntile[0] = P.ntile[1] = P.ntile[2] = 0;
    if (coupled_plan) {
        const size_t elem = fp64_data(prec) ? sizeof(double) : sizeof(float);
        if ((st = ensure_shared(h, &h->dVT, &h->capVT, (size_t)vt_total * elem))) return st;
        // tables: output tiles, per-dimer info, monomer sizes o v, R offsets
        std::vector<CoupDim> cds(D);
        std::vector<int> mdim(N);
        std::vector<long long> rows(N, 0);          // rows each monomer's tiles sum over
        h->r_off.assign(N, 0);
        long long roff = 0;
        for (int m = 0; m < N; m++) {
            mdim[m] = h->mons[m].nocc * (h->mons[m].nao - h->mons[m].nocc);
            h->r_off[m] = roff;
            roff += (long long)mdim[m] * mdim[m];
        }
        long long vt = 0;
        for (int d = 0; d < D; d++) {
            const int X = h->dims[d].X, Y = h->dims[d].Y;
            cds[d] = CoupDim{X, Y, mdim[X], mdim[Y], vt};
            vt += 2LL * cds[d].mX * cds[d].mY;
            rows[X] += mdim[Y];
            rows[Y] += mdim[X];
        }
        // per monomer the tile edge with the least padded upper-triangle work,
        // smaller edges weighted for their extra staging per FMA; within an
        // edge the monomers with the longest sums start first
        static const int kEdge[3] = {64, 48, 32};
        std::vector<int> cls(N), order(N);
        for (int m = 0; m < N; m++) {
            double best = 0;
            for (int c = 0; c < 3; c++) {
                const double nt = (mdim[m] + kEdge[c] - 1) / kEdge[c];
                const double cost = nt * (nt + 1) / 2 * kEdge[c] * kEdge[c] * (1.0 + 16.0 / kEdge[c]);
                if (c == 0 || cost < best) { best = cost; cls[m] = c; }
            }
            order[m] = m;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rows[a] > rows[b]; });
        std::vector<CoupTile> tiles;
        for (int c = 0; c < 3; c++) {
            const size_t before = tiles.size();
            for (int m : order) {
                if (cls[m] != c || mdim[m] == 0) continue;    // a monomer with no dimers gets R = 0
                const int e = kEdge[c];
                for (int p0 = 0; p0 < mdim[m]; p0 += e)
                    for (int q0 = p0; q0 < mdim[m]; q0 += e) tiles.push_back(CoupTile{m, p0, q0});
            }
            P.ntile[c] = (int)(tiles.size() - before);
        }
        std::vector<unsigned char> tab;
        auto put = [&](const void* src, size_t bytes) {
            tab.resize((tab.size() + 15) & ~(size_t)15);
            const size_t off = tab.size();
            tab.resize(off + bytes);
            std::memcpy(tab.data() + off, src, bytes);
            return off;
        };
        P.off_tiles = put(tiles.data(), tiles.size() * sizeof(CoupTile));
        P.off_dims = put(cds.data(), cds.size() * sizeof(CoupDim));
        P.off_mdim = put(mdim.data(), mdim.size() * sizeof(int));
        P.off_roff = put(h->r_off.data(), h->r_off.size() * sizeof(long long));
        // singles term: 256 outputs per tile, monomer blocks of o v
        std::vector<SingTile> stiles;
        std::vector<long long> soff(N + 1, 0);
        for (int m = 0; m < N; m++) {
            soff[m + 1] = soff[m] + mdim[m];
            for (int p0 = 0; p0 < mdim[m]; p0 += 256) stiles.push_back(SingTile{m, p0});
        }
        std::vector<long long> poff(D);
        long long pacc = 0;
        for (int d = 0; d < D; d++) {
            poff[d] = pacc;
            pacc += cds[d].mX + cds[d].mY;
        }
        h->s_total = soff[N];
        h->s_parts = pacc;
        P.nstiles = (int)stiles.size();
        P.off_stiles = put(stiles.data(), stiles.size() * sizeof(SingTile));
        P.off_soff = put(soff.data(), soff.size() * sizeof(long long));
        P.off_poff = put(poff.data(), poff.size() * sizeof(long long));
        if ((st = ensure_shared(h, &h->dCoup, &h->capCoup, tab.size()))) return st;
        if ((st = ensure_shared(h, &h->dR, &h->capR, (size_t)roff * sizeof(double)))) return st;
        CK(h, cudaMemcpyAsync(h->dCoup, tab.data(), tab.size(), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));   // tab is pageable and goes out of scope
    }
    CK(h, cudaMemcpyAsync(P.dDesc, P.hDesc.data(), ndesc * sizeof(DimerDesc), cudaMemcpyHostToDevice, h->stream));
    if (!fold.empty())
        CK(h, cudaMemcpyAsync(P.dFold, fold.data(), fold.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    P.nfold = (int)fold.size() / 3;

    // second-half tasks of the waves with monomers above 32 AO: [tasks][first-task index per dimer]
    std::vector<unsigned char> fin_host;
    std::vector<size_t> fin_off(waves.size(), 0), part_off(waves.size(), 0);
    std::vector<int> ntasks(waves.size(), 0);
    size_t parts = 0;
    for (size_t w = 0; w < waves.size(); w++) {
        const int b = waves[w].first, nd = waves[w].second - b;
        int max_ao = 0;
        for (int k = b; k < b + nd; k++) max_ao = std::max(max_ao, std::max(P.hDesc[k].nX, P.hDesc[k].nY));
        if (max_ao <= 32) continue;
        std::vector<FinTask> t;
        finish_tasks(P.hDesc.data() + b, nd, 1 << 22, &t);
        std::vector<int> first(nd);
        for (size_t q = 0; q < t.size(); q++)
            if (t[q].pr0 == 0) first[t[q].dimer] = (int)q;
        fin_host.resize((fin_host.size() + 255) & ~(size_t)255);
        fin_off[w] = fin_host.size();
        const size_t tb = t.size() * sizeof(FinTask), fb = first.size() * sizeof(int);
        fin_host.resize(fin_host.size() + tb + fb);
        std::memcpy(fin_host.data() + fin_off[w], t.data(), tb);
        std::memcpy(fin_host.data() + fin_off[w] + tb, first.data(), fb);
        ntasks[w] = (int)t.size();
        part_off[w] = parts;
        parts += t.size();
    }
    if (!fin_host.empty()) {
        if ((st = ensure(h, &P.dFin, &P.capFin, fin_host.size()))) return st;
        if ((st = ensure(h, &P.dPart, &P.capPart, parts * 2 * sizeof(double)))) return st;
        CK(h, cudaMemcpyAsync(P.dFin, fin_host.data(), fin_host.size(), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));   // fin_host is pageable and goes out of scope
    }

    for (size_t w = 0; w < waves.size(); w++) {
        mcpt_ctx::Wave wv{};
        wv.b = waves[w].first;
        wv.nd = waves[w].second - wv.b;
        wv.fin_off = fin_off[w];
        wv.ntasks = ntasks[w];
        wv.part_off = part_off[w];
        for (int k = wv.b; k < wv.b + wv.nd; k++) {
            const DimerDesc& dd = P.hDesc[k];
            wv.max_rows = std::max(wv.max_rows, dd.nX * dd.nY);
            wv.max_occ = std::max(wv.max_occ, std::max(dd.oX, dd.oY));
            wv.max_ao = std::max(wv.max_ao, std::max(dd.nX, dd.nY));
        }
        wv.fin_warps = 4;
        if (wv.max_ao <= 32) {
            const int form = prec == MCPT_FP64E ? FIN_FF
                             : fp64_data(prec)  ? FIN_F64
                             : h->fp64_epilogue ? FIN_F32_F64EPI
                                                : FIN_F32_PAIRS;
            wv.fin_warps = finish_w32_warps(P.hDesc.data() + wv.b, wv.nd, form);
        }
        if (is_tensor_form(prec)) {
            char tcerr[256] = {0};
            const size_t end = (w + 1 < work_off.size()) ? work_off[w + 1] : P.capWork;
            const TcKind kind = tc_kind_of(prec);
            void* work = static_cast<char*>(P.dWork) + work_off[w];
            TcTune tune{};
            bool tuned = false;
            if (!h->tune_cache.empty()) {
                tune_load(h);
                const std::string key = tune_key(h, prec, P.hDesc.data() + wv.b, wv.nd);
                auto it = h->tuned.find(key);
                if (it != h->tuned.end()) {
                    tune = it->second;
                } else {
                    float ms = 0;
                    mcpt_status st2 = tune_wave(h, P, kind, wv, work, end - work_off[w], &tune, &ms);
                    if (st2) return st2;
                    h->tuned[key] = tune;
                    std::ofstream out(h->tune_cache, std::ios::app);
                    out << key << ' ' << tune.variant1 << ' ' << tune.sf << ' ' << tune.grid << ' ' << ms / 3
                        << '\n';
                }
                tuned = tune.variant1 != 0;
            }
            cudaError_t e = tc_prepare(kind, P.hDesc.data() + wv.b, P.dDesc + wv.b, wv.nd, h->dCf, h->dC, h->dH, work, end - work_off[w], h->dFlag + 1,
                                       h->stream, tuned ? &tune : nullptr, &wv.tc, tcerr, sizeof tcerr);
            if (e == cudaErrorNotSupported) return fail(h, MCPT_EUNSUPPORTED, "%s", tcerr);
            if (e != cudaSuccess)
                return fail(h, MCPT_ECUDA, "tensor-core plan: %s (%s)", cudaGetErrorString(e), tcerr);
            wv.tc.wait_ns = h->wait_ns;
            wv.tc.withhold = h->withhold;
        }
        P.waves.push_back(wv);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    P.prec = prec;
    P.first = first;
    P.count = count;
    P.alg_bytes = alg_bytes;
    P.alg_flops = alg_flops;
    P.alg_flops_half = alg_flops_half;
    P.valid = true;
    P.epoch = h->epoch;
    return MCPT_OK;
}

// The launch sequence of one run of the current plan on the handle's stream
// (no host synchronisation, no allocation): status reset, then per wave the
// first half and the second half, then the per-monomer reduction.  With `ev`
// (timing), CUDA events are recorded around the phases.
static mcpt_status enqueue_run(mcpt_handle h, const mcpt_ctx::Plan& P, const std::vector<cudaEvent_t>* ev,
                               int* launches_out)
{
    const int D = (int)h->dims.size();
    const int N = (int)h->mons.size();
    const mcpt_precision prec = P.prec;
    const size_t W = P.waves.size();
    CK(h, cudaMemsetAsync(h->dFlag + 1, 0, sizeof(int), h->stream));
    if (ev) CK(h, cudaEventRecord((*ev)[0], h->stream));
    int launches = 0;
    for (size_t w = 0; w < W; w++) {
        const auto& wv = P.waves[w];
        const DimerDesc* wd = P.dDesc + wv.b;
        switch (prec) {
        case MCPT_FP64:
            CK(h, launch_half_fp64(wd, wv.nd, wv.max_rows, wv.max_occ, h->dC, static_cast<double*>(h->dH), h->stream));
            break;
        case MCPT_FP32C:
            CK(h, launch_half_fp32c(wd, wv.nd, wv.max_rows, wv.max_occ, h->dCf, static_cast<float*>(h->dH), h->stream));
            break;
        case MCPT_TF32:
        case MCPT_BF16X3:
        case MCPT_BF16X2:
        case MCPT_FP64E:
            CK(h, tc_launch(wv.tc, h->stream));
            break;
        }
        launches++;
        if (ev) CK(h, cudaEventRecord((*ev)[1 + 2 * w], h->stream));
        const FinTask* tasks =
            wv.ntasks ? reinterpret_cast<const FinTask*>(static_cast<const char*>(P.dFin) + wv.fin_off) : nullptr;
        double* part = wv.ntasks ? P.dPart + 2 * wv.part_off : nullptr;
        if (prec == MCPT_FP64E && wv.max_ao <= 32)   // H as FP32 pairs (the tensor-core launch's h_pairs)
            CK(h, launch_finish_ff(wd, wv.nd, wv.max_ao, h->dC, h->dE, h->dH, h->dE2,
                                   P.coupling ? static_cast<double*>(h->dVT) : nullptr, wv.fin_warps, h->stream));
        else if (fp64_data(prec))
            CK(h, launch_finish_fp64(wd, wv.nd, wv.max_ao, h->dC, h->dE, static_cast<const double*>(h->dH), h->dE2,
                                     tasks, wv.ntasks, part, P.coupling ? static_cast<double*>(h->dVT) : nullptr,
                                     wv.fin_warps, h->stream));
        else
            CK(h, launch_finish_fp32(wd, wv.nd, wv.max_ao, h->dCf, h->dE, static_cast<const float*>(h->dH), h->dE2,
                                     tasks, wv.ntasks, part, P.coupling ? static_cast<float*>(h->dVT) : nullptr,
                                     h->fp64_epilogue, wv.fin_warps, h->stream));
        launches += wv.ntasks ? 2 : 1;
        if (ev) CK(h, cudaEventRecord((*ev)[2 + 2 * w], h->stream));
    }
    if (P.nfold) {
        CK(h, launch_fold(P.dFold, P.nfold, h->dE2, h->stream));
        launches++;
    }
    MonomerLists L{h->dLists, h->dLists + N + 1, N};
    CK(h, launch_reduce(h->dE2, D, L, h->dMon, h->dTot, h->dTot + 2, h->stream));
    if (P.coupling) {
        const char* tab = static_cast<const char*>(h->dCoup);
        const CoupTile* tiles = reinterpret_cast<const CoupTile*>(tab + P.off_tiles);
        const CoupDim* cds = reinterpret_cast<const CoupDim*>(tab + P.off_dims);
        const int* mdim = reinterpret_cast<const int*>(tab + P.off_mdim);
        const long long* roff = reinterpret_cast<const long long*>(tab + P.off_roff);
        if (fp64_data(prec))
            CK(h, launch_coupling_fp64(tiles, P.ntile, cds, L, mdim, roff, static_cast<const double*>(h->dVT), h->dR,
                                       h->stream));
        else
            CK(h, launch_coupling_fp32(tiles, P.ntile, cds, L, mdim, roff, static_cast<const float*>(h->dVT), h->dR,
                                       h->stream));
        launches += (P.ntile[0] > 0) + (P.ntile[1] > 0) + (P.ntile[2] > 0);
    }
    launches += 2;   // the reduction: partial sums, then their merge
    if (ev) CK(h, cudaEventRecord((*ev)[2 * W + 1], h->stream));
    *launches_out = launches;
    return MCPT_OK;
}

// Plans kept per context; beyond this the least recently used is rebuilt.
constexpr size_t kMaxPlans = 64;

// The plan of (first, count, precision): a cached one that is still valid,
// else one (re)built, reusing the stale entry of the same key or the least
// recently used slot.
static mcpt_status get_plan(mcpt_handle h, int first, int count, mcpt_ctx::Plan** out)
{
    mcpt_ctx::Plan* hit = nullptr;
    for (auto& p : h->plans)
        if (p->first == first && p->count == count && p->prec == h->prec && (p->valid || !hit)) {
            hit = p.get();
            if (p->valid) break;
        }
    if (!hit || !hit->valid || hit->epoch != h->epoch) {
        if (!hit) {
            if (h->plans.size() < kMaxPlans) {
                h->plans.emplace_back(new mcpt_ctx::Plan());
                hit = h->plans.back().get();
            } else {
                hit = h->plans[0].get();
                for (auto& p : h->plans)
                    if (p->last_use < hit->last_use) hit = p.get();
                CK(h, cudaStreamSynchronize(h->stream));   // its buffers may still be in use
                if (h->coup == hit) h->coup = nullptr;
            }
        }
        if (hit->graph) {
            CK(h, cudaStreamSynchronize(h->stream));
            cudaGraphExecDestroy(hit->graph);
            hit->graph = nullptr;
        }
        hit->prec = h->prec;
        hit->first = first;
        hit->count = count;
        mcpt_status st = build_plan(h, *hit, first, count);
        if (st) {
            hit->valid = false;
            return st;
        }
    }
    hit->last_use = ++h->use_clock;
    *out = hit;
    return MCPT_OK;
}

static mcpt_status run_impl(mcpt_handle h, int first, int count)
{
    CK(h, cudaSetDevice(h->device));
    mcpt_ctx::Plan* Pp = nullptr;
    mcpt_status pst = get_plan(h, first, count, &Pp);
    if (pst) return pst;
    auto& P = *Pp;
    RunEvents& re = h->rev;
    const size_t W = P.waves.size();
    int launches = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(h, cudaStreamIsCapturing(h->stream, &cap));
    if (h->timing) {
        std::vector<cudaEvent_t> ev;
        while (ev.size() < 2 + 2 * W) {
            if (!re.pool.empty()) {
                ev.push_back(re.pool.back());
                re.pool.pop_back();
            } else {
                cudaEvent_t e;
                CK(h, cudaEventCreate(&e));
                ev.push_back(e);
            }
        }
        mcpt_status st = enqueue_run(h, P, &ev, &launches);
        re.pending.push_back(std::move(ev));
        if (st) return st;
    } else if (h->graphs && cap == cudaStreamCaptureStatusNone) {
        // replay the plan's launches as one CUDA graph (captured on first use)
        if (!P.graph) {
            CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
            mcpt_status st = enqueue_run(h, P, nullptr, &launches);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            CK(h, e);
            e = cudaGraphInstantiate(&P.graph, g, 0);
            cudaGraphDestroy(g);
            CK(h, e);
            P.graph_launches = launches;
        }
        CK(h, cudaGraphLaunch(P.graph, h->stream));
        launches = P.graph_launches;
    } else {
        mcpt_status st = enqueue_run(h, P, nullptr, &launches);
        if (st) return st;
    }

    for (int k = 0; k < count; k++) h->dims[first + k].computed = true;
    re.runs++;
    re.launches += launches;
    h->stats.waves = (int)W;
    h->stats.alg_bytes = P.alg_bytes;
    h->stats.alg_flops = P.alg_flops;
    h->stats.alg_flops_half = P.alg_flops_half;
    h->ran = true;
    h->coupled = P.coupling;
    if (P.coupling) h->coup = &P;
    return MCPT_OK;
}

mcpt_status mcpt_run(mcpt_handle h)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_run: NULL handle");
    if (h->dims.empty()) return fail(h, MCPT_ESTATE, "mcpt_run: no dimers registered");
    return run_impl(h, 0, (int)h->dims.size());
}

mcpt_status mcpt_run_range(mcpt_handle h, int first, int count)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_run_range: NULL handle");
    const int D = (int)h->dims.size();
    if (D == 0) return fail(h, MCPT_ESTATE, "mcpt_run_range: no dimers registered");
    if (first < 0 || count < 1 || first + count > D)
        return fail(h, MCPT_EINVAL, "mcpt_run_range: [%d, %d) outside [0, %d)", first, first + count, D);
    return run_impl(h, first, count);
}

mcpt_status mcpt_energies(mcpt_handle h, double* mon_J, double* mon_K, double* per_dimer, double* total)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_energies: NULL handle");
    if (!h->ran) return fail(h, MCPT_ESTATE, "mcpt_energies: no run yet");
    for (size_t d = 0; d < h->dims.size(); d++)
        if (!h->dims[d].computed)
            return fail(h, MCPT_ESTATE, "mcpt_energies: dimer %zu has not been computed since it was added", d);
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    int status = 0;
    CK(h, cudaMemcpy(&status, h->dFlag + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (status)
        return fail(h, MCPT_ETIMEOUT, "mcpt_energies: a device-side wait gave up (status 0x%x)", status);
    const int N = (int)h->mons.size(), D = (int)h->dims.size();
    if (mon_J) CK(h, cudaMemcpy(mon_J, h->dMon, N * sizeof(double), cudaMemcpyDeviceToHost));
    if (mon_K) CK(h, cudaMemcpy(mon_K, h->dMon + N, N * sizeof(double), cudaMemcpyDeviceToHost));
    if (per_dimer) CK(h, cudaMemcpy(per_dimer, h->dE2, 2 * (size_t)D * sizeof(double), cudaMemcpyDeviceToHost));
    if (total) CK(h, cudaMemcpy(total, h->dTot, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    return MCPT_OK;
}

mcpt_status mcpt_coupling(mcpt_handle h, int X, double* R)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_coupling: NULL handle");
    if (X < 0 || X >= (int)h->mons.size())
        return fail(h, MCPT_EINVAL, "mcpt_coupling: unknown monomer %d of %zu", X, h->mons.size());
    if (!R) return fail(h, MCPT_EINVAL, "mcpt_coupling: R is NULL");
    if (!h->coupling) return fail(h, MCPT_ESTATE, "mcpt_coupling: the context was created with coupling = 0");
    if (!h->coupled)
        return fail(h, MCPT_ESTATE, "mcpt_coupling: no mcpt_run of every dimer since the integrals last changed");
    CK(h, cudaSetDevice(h->device));
    const size_t mm = (size_t)h->mons[X].nocc * (h->mons[X].nao - h->mons[X].nocc);
    CK(h, cudaStreamSynchronize(h->stream));
    int status = 0;
    CK(h, cudaMemcpy(&status, h->dFlag + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) return fail(h, MCPT_ETIMEOUT, "mcpt_coupling: a device-side wait gave up (status 0x%x)", status);
    CK(h, cudaMemcpy(R, h->dR + h->r_off[X], mm * mm * sizeof(double), cudaMemcpyDeviceToHost));
    return MCPT_OK;
}

mcpt_status mcpt_singles(mcpt_handle h, const double* t, double* s)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_singles: NULL handle");
    if (!t || !s) return fail(h, MCPT_EINVAL, "mcpt_singles: t or s is NULL");
    if (!h->coupling) return fail(h, MCPT_ESTATE, "mcpt_singles: the context was created with coupling = 0");
    if (!h->coupled)
        return fail(h, MCPT_ESTATE, "mcpt_singles: no mcpt_run of every dimer since the integrals last changed");
    if (!h->coup) return fail(h, MCPT_ESTATE, "mcpt_singles: no coupling plan");
    const mcpt_ctx::Plan& P = *h->coup;
    const size_t M = (size_t)h->s_total;
    if (h->validate && !all_finite(t, M)) return fail(h, MCPT_EINVAL, "mcpt_singles: t has a non-finite value");
    if (M == 0) return MCPT_OK;
    CK(h, cudaSetDevice(h->device));
    mcpt_status st;
    if ((st = ensure(h, &h->dS1, &h->capS1, (2 * M + (size_t)h->s_parts) * sizeof(double)))) return st;
    CK(h, cudaMemcpyAsync(h->dS1, t, M * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const char* tab = static_cast<const char*>(h->dCoup);
    const SingTile* tiles = reinterpret_cast<const SingTile*>(tab + P.off_stiles);
    const CoupDim* cds = reinterpret_cast<const CoupDim*>(tab + P.off_dims);
    const int* mdim = reinterpret_cast<const int*>(tab + P.off_mdim);
    const long long* soff = reinterpret_cast<const long long*>(tab + P.off_soff);
    const long long* poff = reinterpret_cast<const long long*>(tab + P.off_poff);
    const int N = (int)h->mons.size(), D = (int)h->dims.size();
    MonomerLists L{h->dLists, h->dLists + N + 1, N};
    double* part = h->dS1 + 2 * M;
    if (fp64_data(P.prec))
        CK(h, launch_singles_fp64(tiles, P.nstiles, cds, D, L, mdim, soff, poff, static_cast<const double*>(h->dVT),
                                  h->dS1, part, h->dS1 + M, h->stream));
    else
        CK(h, launch_singles_fp32(tiles, P.nstiles, cds, D, L, mdim, soff, poff, static_cast<const float*>(h->dVT),
                                  h->dS1, part, h->dS1 + M, h->stream));
    CK(h, cudaMemcpyAsync(s, h->dS1 + M, M * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    int status = 0;
    CK(h, cudaMemcpy(&status, h->dFlag + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) return fail(h, MCPT_ETIMEOUT, "mcpt_singles: a device-side wait gave up (status 0x%x)", status);
    return MCPT_OK;
}

mcpt_status mcpt_add_dimer_df(mcpt_handle h, int X, int Y, const double* B, int naux, double s, int on_device,
                              int* id_out)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_add_dimer_df: NULL handle");
    const int N = (int)h->mons.size();
    if (X < 0 || X >= N || Y < 0 || Y >= N)
        return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: unknown monomer id (%d, %d) of %d", X, Y, N);
    if (X >= Y) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: factors must be given with X < Y (%d, %d)", X, Y);
    if (!B) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: B is NULL");
    if (naux < 1) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: naux=%d < 1", naux);
    if (!std::isfinite(s)) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: s is not finite");
    const std::pair<int, int> key(X, Y);
    if (h->df_pairs.count(key)) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: duplicate dimer (%d, %d)", X, Y);
    const int n = h->mons[X].nao + h->mons[Y].nao;
    const size_t elems = (size_t)naux * n * n;
    CK(h, cudaSetDevice(h->device));
    DfRec r{X, Y, B, naux, s};
    mcpt_status st;
    if (on_device) {
        if ((st = check_device_ptr(h, B, "mcpt_add_dimer_df"))) return st;
        if (h->validate) {
            CK(h, cudaMemsetAsync(h->dFlag, 0, sizeof(int), h->stream));
            CK(h, launch_check_finite(B, (long long)elems, h->dFlag, h->stream));
            int flag = 0;
            CK(h, cudaMemcpyAsync(&flag, h->dFlag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            if (flag) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: non-finite factor");
        }
    } else {
        if (h->validate && !all_finite(B, elems)) return fail(h, MCPT_EINVAL, "mcpt_add_dimer_df: non-finite factor");
        void* dst = nullptr;
        if ((st = arena_alloc(h, elems * sizeof(double), &dst))) return st;
        CK(h, cudaMemcpyAsync(dst, B, elems * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        r.B = static_cast<const double*>(dst);
    }
    h->dfs.push_back(r);
    h->df_pairs.insert(key);
    h->df_ran = false;
    if (id_out) *id_out = (int)h->dfs.size() - 1;
    return MCPT_OK;
}

mcpt_status mcpt_run_df(mcpt_handle h)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_run_df: NULL handle");
    const int N = (int)h->mons.size(), D = (int)h->dfs.size();
    if (D == 0) return fail(h, MCPT_ESTATE, "mcpt_run_df: no density-fitted dimers registered");
    CK(h, cudaSetDevice(h->device));
    mcpt_status st = upload_static(h);
    if (st) return st;
    const bool fp64 = fp64_data(h->prec);
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    std::vector<DfDim> dims(D);
    long long hoff = 0;
    int poff = 0, max_naux = 0, max_pairs = 0, max_on = 0, max_v = 0;
    for (int d = 0; d < D; d++) {
        const DfRec& r = h->dfs[d];
        const MonomerRec& mX = h->mons[r.X];
        const MonomerRec& mY = h->mons[r.Y];
        const int nX = mX.nao, nY = mY.nao, oX = mX.nocc, oY = mY.nocc, vX = nX - oX, vY = nY - oY;
        // shared memory of the half-transformation: B^Q, C_X, C_Y and the occupied rows
        const int on = (nX + nY) * (nX + nY) + nX * nX + nY * nY + (oX + oY) * (nX + nY);
        if ((size_t)on * es > (size_t)200 * 1024)
            return fail(h, MCPT_EUNSUPPORTED, "mcpt_run_df: dimer %d (%d + %d AO) needs %zu bytes of shared memory",
                        d, nX, nY, (size_t)on * es);
        dims[d] = DfDim{r.B, r.naux, nX, nY, oX, oY, mX.offC, mY.offC, mX.offE, mY.offE, r.s, hoff, poff, d};
        hoff += (long long)r.naux * ((long long)oX * vX + (long long)oY * vY + (long long)oX * vY + (long long)oY * vX);
        hoff = (hoff + 63) / 64 * 64;
        poff += oX * oY;
        max_naux = std::max(max_naux, r.naux);
        max_pairs = std::max(max_pairs, oX * oY);
        max_on = std::max(max_on, on);
        max_v = std::max(max_v, std::max(vX, vY));
    }
    // monomer lists of the density-fitted dimers (CSR, ascending dimer id)
    std::vector<int> cnt(N + 1, 0), lists(N + 1 + 2 * (size_t)D);
    for (const auto& r : h->dfs) { cnt[r.X + 1]++; cnt[r.Y + 1]++; }
    for (int m = 0; m < N; m++) cnt[m + 1] += cnt[m];
    std::copy(cnt.begin(), cnt.end(), lists.begin());
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int d = 0; d < D; d++) {
        lists[N + 1 + fill[h->dfs[d].X]++] = d;
        lists[N + 1 + fill[h->dfs[d].Y]++] = d;
    }
    // scratch: table, half-transformed blocks, pair partials
    const size_t tab = ((size_t)D * sizeof(DfDim) + 255) & ~(size_t)255;
    const size_t halfb = ((size_t)hoff * es + 255) & ~(size_t)255;
    const size_t partb = 2 * (size_t)poff * sizeof(double);
    if ((st = ensure(h, &h->dDf, &h->capDf, tab + halfb + partb))) return st;
    if ((st = ensure(h, &h->dDfOut, &h->capDfOut,
                     (2 * (size_t)D + 2 * (size_t)N + 2 + 4 * kReduceBlocks) * sizeof(double))))
        return st;
    if ((st = ensure(h, &h->dDfLists, &h->capDfLists, lists.size() * sizeof(int)))) return st;
    char* base = static_cast<char*>(h->dDf);
    CK(h, cudaMemcpyAsync(base, dims.data(), (size_t)D * sizeof(DfDim), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->dDfLists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    double* E2 = h->dDfOut;
    CK(h, launch_df(fp64, reinterpret_cast<const DfDim*>(base), D, max_naux, max_pairs, max_on, max_v, h->dC, h->dE,
                    base + tab, reinterpret_cast<double*>(base + tab + halfb), E2, h->stream));
    MonomerLists L{h->dDfLists, h->dDfLists + N + 1, N};
    CK(h, launch_reduce(E2, D, L, E2 + 2 * (size_t)D, E2 + 2 * (size_t)D + 2 * (size_t)N,
                        E2 + 2 * (size_t)D + 2 * (size_t)N + 2, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));   // the host tables go out of scope
    h->df_ran = true;
    return MCPT_OK;
}

mcpt_status mcpt_df_energies(mcpt_handle h, double* mon_J, double* mon_K, double* per_dimer, double* total)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_df_energies: NULL handle");
    if (!h->df_ran) return fail(h, MCPT_ESTATE, "mcpt_df_energies: no mcpt_run_df since the last dimer was added");
    const int N = (int)h->mons.size(), D = (int)h->dfs.size();
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    const double* E2 = h->dDfOut;
    if (mon_J) CK(h, cudaMemcpy(mon_J, E2 + 2 * (size_t)D, N * sizeof(double), cudaMemcpyDeviceToHost));
    if (mon_K) CK(h, cudaMemcpy(mon_K, E2 + 2 * (size_t)D + N, N * sizeof(double), cudaMemcpyDeviceToHost));
    if (per_dimer) CK(h, cudaMemcpy(per_dimer, E2, 2 * (size_t)D * sizeof(double), cudaMemcpyDeviceToHost));
    if (total) CK(h, cudaMemcpy(total, E2 + 2 * (size_t)D + 2 * (size_t)N, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    return MCPT_OK;
}

mcpt_status mcpt_set_monomer_doubles(mcpt_handle h, int X, const double* G, const double* U)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_set_monomer_doubles: NULL handle");
    if (X < 0 || X >= (int)h->mons.size())
        return fail(h, MCPT_EINVAL, "mcpt_set_monomer_doubles: unknown monomer %d of %zu", X, h->mons.size());
    const size_t m = (size_t)h->mons[X].nocc * (h->mons[X].nao - h->mons[X].nocc);
    if (h->validate && ((G && !all_finite(G, m * m)) || (U && !all_finite(U, m * m))))
        return fail(h, MCPT_EINVAL, "mcpt_set_monomer_doubles: non-finite value");
    h->monG.resize(h->mons.size());
    h->monU.resize(h->mons.size());
    h->monG[X] = G ? std::vector<double>(G, G + m * m) : std::vector<double>();
    h->monU[X] = U ? std::vector<double>(U, U + m * m) : std::vector<double>();
    return MCPT_OK;
}

}  // extern "C"

namespace {

template <typename T>
struct Td2Tables {
    std::vector<Td2Dim> dims;
    std::vector<long long> goff, wdoff;
    std::vector<QStep<double, T>> q1[2];        // first steps (FP64 AO input) of K and A
    std::vector<QStep<T, T>> q[2][3];          // steps 2-4 of K and A
    std::vector<PGemm<T>> pg[8];               // source X, source Y, terms L1..L6
    int maxM[2][4] = {{0}}, maxN[2][4] = {{0}}, maxR[8] = {0}, maxC[8] = {0};
    int maxE = 0, maxVV = 0;
};

inline PAxis ax(int n1, long long s0, long long s1) { return PAxis{n1 > 0 ? n1 : 1, s0, s1}; }

template <typename T>
mcpt_status td2_run(mcpt_handle h, int n_iter, double* per_dimer, double* delta)
{
    const int N = (int)h->mons.size(), D = (int)h->dims.size();
    mcpt_status st = upload_static(h);
    if (st) return st;
    // monomer matrices in the arithmetic type, G then U per monomer that has them
    h->monG.resize(N);
    h->monU.resize(N);
    std::vector<long long> gOff(N, -1), uOff(N, -1);
    std::vector<T> pool;
    for (int m = 0; m < N; m++) {
        if (!h->monG[m].empty()) { gOff[m] = (long long)pool.size(); pool.insert(pool.end(), h->monG[m].begin(), h->monG[m].end()); }
        if (!h->monU[m].empty()) { uOff[m] = (long long)pool.size(); pool.insert(pool.end(), h->monU[m].begin(), h->monU[m].end()); }
    }
    const T* dMon = nullptr;
    if (!pool.empty()) {
        if ((st = ensure(h, &h->dTd2Mon, &h->capTd2Mon, pool.size() * sizeof(T)))) return st;
        CK(h, cudaMemcpyAsync(h->dTd2Mon, pool.data(), pool.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
        dMon = static_cast<const T*>(h->dTd2Mon);
    }
    // outputs: 2 D energies, then n_iter 8-byte slots of max |dT| bits
    const size_t outBytes = (2 * (size_t)D + (size_t)n_iter) * sizeof(double);
    if ((st = ensure(h, &h->dTd2Out, &h->capTd2Out, outBytes))) return st;
    double* dE = static_cast<double*>(h->dTd2Out);
    unsigned long long* dDelta = reinterpret_cast<unsigned long long*>(dE + 2 * (size_t)D);
    CK(h, cudaMemsetAsync(dDelta, 0, (size_t)n_iter * sizeof(unsigned long long), h->stream));
    const size_t budget = std::max(h->wave_bytes, (size_t)4 << 30);
    auto round64 = [](long long x) { return (x + 63) / 64 * 64; };
    int b0 = 0;
    while (b0 < D) {
        // ---- the batch: consecutive dimers under the budget
        long long tot[9] = {0};            // sections: g, s0, s1, V, W, R0, R, Tc, packed ladder
        int b1 = b0;
        while (b1 < D && b1 - b0 < 65535) {
            const MonomerRec& mX = h->mons[h->dims[b1].X];
            const MonomerRec& mY = h->mons[h->dims[b1].Y];
            const long long big = round64((long long)mX.nao * mX.nao * mY.nao * mY.nao);
            const long long sm = round64((long long)mX.nocc * (mX.nao - mX.nocc) * mY.nocc * (mY.nao - mY.nocc));
            const long long vv = (long long)(mX.nao - mX.nocc) * (mY.nao - mY.nocc);
            const long long lad = round64(vv * ((vv + 3) / 4 * 4));
            const long long need = (3 * big + 5 * sm + lad) * (long long)sizeof(T);
            long long cur = 0;
            for (int k = 0; k < 9; k++) cur += tot[k];
            if (b1 > b0 && (size_t)(cur * (long long)sizeof(T) + need) > budget) break;
            for (int k = 0; k < 3; k++) tot[k] += big;
            for (int k = 3; k < 8; k++) tot[k] += sm;
            tot[8] += lad;
            b1++;
        }
        const int nb = b1 - b0;
        long long sec[9], acc = 0;
        for (int k = 0; k < 9; k++) { sec[k] = acc; acc += tot[k]; }
        if ((st = ensure(h, &h->dTd2, &h->capTd2, (size_t)acc * sizeof(T)))) return st;
        T* arena = static_cast<T*>(h->dTd2);
        // ---- tables
        Td2Tables<T> tb;
        long long run[9];
        for (int k = 0; k < 9; k++) run[k] = sec[k];
        for (int d = b0; d < b1; d++) {
            const DimerRec& r = h->dims[d];
            const MonomerRec& mX = h->mons[r.X];
            const MonomerRec& mY = h->mons[r.Y];
            const int nX = mX.nao, nY = mY.nao, oX = mX.nocc, oY = mY.nocc, vX = nX - oX, vY = nY - oY;
            const long long mXl = (long long)oX * vX, mYl = (long long)oY * vY;
            const long long big = round64((long long)nX * nX * nY * nY), sm = round64(mXl * mYl);
            const int vv = vX * vY, ldw = (vv + 3) / 4 * 4;
            const long long g = run[0], s0 = run[1], s1 = run[2], wd = run[8];
            Td2Dim td{nX, nY, oX, oY, mX.offE, mY.offE, run[3], run[4], run[5], run[6], run[7]};
            for (int k = 0; k < 3; k++) run[k] += big;
            for (int k = 3; k < 8; k++) run[k] += sm;
            run[8] += round64((long long)vv * ldw);
            tb.dims.push_back(td);
            tb.goff.push_back(g);
            tb.wdoff.push_back(wd);
            tb.maxVV = std::max(tb.maxVV, vv);
            const double* CX = h->dC + mX.offC;
            const double* CY = h->dC + mY.offC;
            // K[mu][lam][sig][nu]: nu -> a, sig -> j, lam -> b, mu -> i  => W[i][b][j][a]
            tb.q1[0].push_back(QStep<double, T>{r.E[1], r.st[1][0], r.st[1][1], r.st[1][2], nY, nY, CX, nX, oX,
                                                nX * nY * nY, vX, nX, arena + s0});
            tb.q[0][0].push_back(QStep<T, T>{arena + s0, nY, 0, 0, 1, 1, CY, nY, 0, vX * nX * nY, oY, nY, arena + s1});
            tb.q[0][1].push_back(QStep<T, T>{arena + s1, nY, 0, 0, 1, 1, CY, nY, oY, oY * vX * nX, vY, nY, arena + s0});
            tb.q[0][2].push_back(QStep<T, T>{arena + s0, nX, 0, 0, 1, 1, CX, nX, 0, vY * oY * vX, oX, nX, arena + td.W});
            // A[mu][nu][lam][sig]: sig, lam, nu, mu -> all MOs  => g[p][q][r][s]
            tb.q1[1].push_back(QStep<double, T>{r.E[0], r.st[0][0], r.st[0][1], r.st[0][2], nX, nY, CY, nY, 0,
                                                nX * nX * nY, nY, nY, arena + s0});
            tb.q[1][0].push_back(QStep<T, T>{arena + s0, nY, 0, 0, 1, 1, CY, nY, 0, nY * nX * nX, nY, nY, arena + s1});
            tb.q[1][1].push_back(QStep<T, T>{arena + s1, nX, 0, 0, 1, 1, CX, nX, 0, nY * nY * nX, nX, nX, arena + s0});
            tb.q[1][2].push_back(QStep<T, T>{arena + s0, nX, 0, 0, 1, 1, CX, nX, 0, nX * nY * nY, nX, nX, arena + g});
            const int Mk[4] = {nX * nY * nY, vX * nX * nY, oY * vX * nX, vY * oY * vX};
            const int Nk[4] = {vX, oY, vY, oX};
            const int Ma[4] = {nX * nX * nY, nY * nX * nX, nY * nY * nX, nX * nY * nY};
            const int Na[4] = {nY, nY, nX, nX};
            for (int k = 0; k < 4; k++) {
                tb.maxM[0][k] = std::max(tb.maxM[0][k], Mk[k]);
                tb.maxN[0][k] = std::max(tb.maxN[0][k], Nk[k]);
                tb.maxM[1][k] = std::max(tb.maxM[1][k], Ma[k]);
                tb.maxN[1][k] = std::max(tb.maxN[1][k], Na[k]);
            }
            tb.maxE = std::max(tb.maxE, (int)(mXl * mYl));
            // strides: amplitudes [i][a][j][b], g [p][q][r][s]
            const long long si = vX * mYl, sa = mYl, sj = vY, sb = 1;
            const long long sp = (long long)nX * nY * nY, sq = (long long)nY * nY, sr = nY, ss = 1;
            T* Gb = arena + g;
            T* Tc = arena + td.Tc;
            T* R = arena + td.R;
            T* R0 = arena + td.R0;
            T* V = arena + td.V;
            const int iX = (int)mXl, iY = (int)mYl;
            PGemm<T> none{};
            none.wr = none.wk = none.zk = none.zc = none.orow = none.ocol = ax(1, 0, 0);
            // sources: U_X V and V U_Y^T into R0
            PGemm<T> sx = none, sy = none;
            if (uOff[r.X] >= 0)
                sx = PGemm<T>{dMon + uOff[r.X], ax(iX, 0, iX), ax(iX, 0, 1), V, ax(iX, 0, iY), ax(iY, 0, 1),
                              R0, ax(iX, 0, iY), ax(iY, 0, 1), iX, iY, iX, T(1)};
            if (uOff[r.Y] >= 0)
                sy = PGemm<T>{dMon + uOff[r.Y], ax(iY, 0, iY), ax(iY, 0, 1), V, ax(iY, 0, 1), ax(iX, 0, iY),
                              R0, ax(iY, 0, 1), ax(iX, 0, iY), iY, iX, iY, T(1)};
            // L1 particle ladder: R[(a,b)][(i,j)] += Wt[(a1,b1)][(a,b)] T[(a1,b1)][(i,j)], Wt the
            // packed g[oX+a][oX+a1][oY+b][oY+b1] (k-major, dense rows of ldw)
            PGemm<T> l1{arena + wd, ax(vv, 0, ldw), ax(1, 0, 1),
                        Tc, ax(vY, sa, sb), ax(oY, si, sj), R, ax(vY, sa, sb), ax(oY, si, sj),
                        vv, oX * oY, vv, T(1)};
            // L2 hole ladder: R[(i,j)][(a,b)] += g[i1][i][j1][j] T[(i1,j1)][(a,b)]
            PGemm<T> l2{Gb, ax(oY, sq, ss), ax(oY, sp, sr), Tc, ax(oY, si, sj), ax(vY, sa, sb),
                        R, ax(oY, si, sj), ax(vY, sa, sb), oX * oY, vX * vY, oX * oY, T(1)};
            // L3: R[(i,b)][(a,j)] -= g[i1][i][oY+b][oY+b1] T[(i1,b1)][(a,j)]
            PGemm<T> l3{Gb + oY * sr + oY * ss, ax(vY, sq, sr), ax(vY, sp, ss), Tc, ax(vY, si, sb), ax(oY, sa, sj),
                        R, ax(vY, si, sb), ax(oY, sa, sj), oX * vY, vX * oY, oX * vY, T(-1)};
            // L4: R[(a,j)][(i,b)] -= g[oX+a][oX+a1][j1][j] T[(a1,j1)][(i,b)]
            PGemm<T> l4{Gb + oX * sp + oX * sq, ax(oY, sp, ss), ax(oY, sq, sr), Tc, ax(oY, sa, sj), ax(vY, si, sb),
                        R, ax(oY, sa, sj), ax(vY, si, sb), vX * oY, oX * vY, vX * oY, T(-1)};
            // L5, L6: monomer ring matrices
            PGemm<T> l5 = none, l6 = none;
            if (gOff[r.X] >= 0)
                l5 = PGemm<T>{dMon + gOff[r.X], ax(iX, 0, iX), ax(iX, 0, 1), Tc, ax(iX, 0, iY), ax(iY, 0, 1),
                              R, ax(iX, 0, iY), ax(iY, 0, 1), iX, iY, iX, T(1)};
            if (gOff[r.Y] >= 0)
                l6 = PGemm<T>{dMon + gOff[r.Y], ax(iY, 0, iY), ax(iY, 0, 1), Tc, ax(iY, 0, 1), ax(iX, 0, iY),
                              R, ax(iY, 0, 1), ax(iX, 0, iY), iY, iX, iY, T(1)};
            const PGemm<T> all[8] = {sx, sy, l1, l2, l3, l4, l5, l6};
            for (int k = 0; k < 8; k++) {
                tb.pg[k].push_back(all[k]);
                tb.maxR[k] = std::max(tb.maxR[k], all[k].R);
                tb.maxC[k] = std::max(tb.maxC[k], all[k].C);
            }
        }
        // ---- upload the tables (one buffer, 16-byte aligned pieces)
        std::vector<unsigned char> tab;
        auto put = [&](const void* src, size_t bytes) {
            tab.resize((tab.size() + 15) & ~(size_t)15);
            const size_t off = tab.size();
            tab.resize(off + bytes);
            std::memcpy(tab.data() + off, src, bytes);
            return off;
        };
        const size_t oDims = put(tb.dims.data(), nb * sizeof(Td2Dim));
        const size_t oG = put(tb.goff.data(), nb * sizeof(long long));
        const size_t oWd = put(tb.wdoff.data(), nb * sizeof(long long));
        size_t oQ1[2], oQ[2][3], oP[8];
        for (int f = 0; f < 2; f++) {
            oQ1[f] = put(tb.q1[f].data(), nb * sizeof(QStep<double, T>));
            for (int k = 0; k < 3; k++) oQ[f][k] = put(tb.q[f][k].data(), nb * sizeof(QStep<T, T>));
        }
        for (int k = 0; k < 8; k++) oP[k] = put(tb.pg[k].data(), nb * sizeof(PGemm<T>));
        if ((st = ensure(h, &h->dTd2Tab, &h->capTd2Tab, tab.size()))) return st;
        CK(h, cudaMemcpyAsync(h->dTd2Tab, tab.data(), tab.size(), cudaMemcpyHostToDevice, h->stream));
        const unsigned char* tbase = static_cast<const unsigned char*>(h->dTd2Tab);
        auto at = [&](size_t off) { return static_cast<const void*>(tbase + off); };
        const Td2Dim* dDims = static_cast<const Td2Dim*>(at(oDims));
        // ---- transformations: K (W), then A (g)
        for (int f = 0; f < 2; f++) {
            CK(h, launch_qstep(static_cast<const QStep<double, T>*>(at(oQ1[f])), nb, tb.maxM[f][0], tb.maxN[f][0],
                               h->stream));
            for (int k = 0; k < 3; k++)
                CK(h, launch_qstep(static_cast<const QStep<T, T>*>(at(oQ[f][k])), nb, tb.maxM[f][k + 1],
                                   tb.maxN[f][k + 1], h->stream));
        }
        CK(h, launch_td2_init<T>(dDims, static_cast<const long long*>(at(oG)), nb, tb.maxE, arena, h->stream));
        CK(h, launch_pack_ladder<T>(dDims, static_cast<const long long*>(at(oG)), static_cast<const long long*>(at(oWd)),
                                    nb, tb.maxVV, arena, h->stream));
        for (int k = 0; k < 2; k++)
            CK(h, launch_pgemm(static_cast<const PGemm<T>*>(at(oP[k])), nb, tb.maxR[k], tb.maxC[k], h->stream));
        // ---- Jacobi steps
        for (int it = 0; it < n_iter; it++) {
            CK(h, cudaMemcpyAsync(arena + sec[6], arena + sec[5], (size_t)tot[5] * sizeof(T),
                                  cudaMemcpyDeviceToDevice, h->stream));
            CK(h, launch_pgemm_dw(static_cast<const PGemm<T>*>(at(oP[2])), nb, tb.maxR[2], tb.maxC[2], h->stream));
            for (int k = 3; k < 8; k++)
                CK(h, launch_pgemm(static_cast<const PGemm<T>*>(at(oP[k])), nb, tb.maxR[k], tb.maxC[k], h->stream));
            CK(h, launch_td2_update<T>(dDims, nb, tb.maxE, h->dE, arena, dDelta + it, h->stream));
        }
        CK(h, launch_td2_energy<T>(dDims, nb, arena, dE + 2 * (size_t)b0, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));        // the tables are reused by the next batch
        b0 = b1;
    }
    std::vector<unsigned long long> bits(n_iter);
    if (per_dimer) CK(h, cudaMemcpy(per_dimer, dE, 2 * (size_t)D * sizeof(double), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(bits.data(), dDelta, (size_t)n_iter * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    if (delta)
        for (int it = 0; it < n_iter; it++) {
            if (sizeof(T) == 4) {
                const unsigned int u = (unsigned int)(bits[it] & 0xffffffffu);
                float f;
                std::memcpy(&f, &u, sizeof f);
                delta[it] = f;
            } else {
                std::memcpy(&delta[it], &bits[it], sizeof(double));
            }
        }
    return MCPT_OK;
}

}  // namespace

extern "C" {

mcpt_status mcpt_td2(mcpt_handle h, int n_iter, double* per_dimer, double* delta)
{
    if (!h) return fail(nullptr, MCPT_EINVAL, "mcpt_td2: NULL handle");
    if (n_iter < 1 || n_iter > 10000) return fail(h, MCPT_EINVAL, "mcpt_td2: n_iter=%d outside [1, 10000]", n_iter);
    if (h->dims.empty()) return fail(h, MCPT_ESTATE, "mcpt_td2: no dimers registered");
    CK(h, cudaSetDevice(h->device));
    return fp64_data(h->prec) ? td2_run<double>(h, n_iter, per_dimer, delta)
                                : td2_run<float>(h, n_iter, per_dimer, delta);
}

mcpt_status mcpt_collect_stats(mcpt_handle h, mcpt_run_stats* out)
{
    if (!h || !out) return fail(h, MCPT_EINVAL, "mcpt_collect_stats: NULL argument");
    if (!h->ran) return fail(h, MCPT_ESTATE, "mcpt_collect_stats: no run yet");
    CK(h, cudaSetDevice(h->device));
    *out = h->stats;
    for (int k = 0; k < 4; k++) out->ms[k] = 0.f;
    RunEvents& re = h->rev;
    out->runs = re.runs;
    out->launches = re.launches;
    if (!re.pending.empty()) {
        CK(h, cudaStreamSynchronize(h->stream));
        for (auto& ev : re.pending) {
            const int W = (int)(ev.size() - 2) / 2;
            float t;
            for (int w = 0; w < W; w++) {
                CK(h, cudaEventElapsedTime(&t, ev[2 * w], ev[1 + 2 * w]));
                out->ms[0] += t;
                CK(h, cudaEventElapsedTime(&t, ev[1 + 2 * w], ev[2 + 2 * w]));
                out->ms[1] += t;
            }
            CK(h, cudaEventElapsedTime(&t, ev[2 * W], ev[2 * W + 1]));
            out->ms[2] += t;
            CK(h, cudaEventElapsedTime(&t, ev[0], ev[2 * W + 1]));
            out->ms[3] += t;
            re.pool.insert(re.pool.end(), ev.begin(), ev.end());
        }
        re.pending.clear();
    }
    re.runs = 0;
    re.launches = 0;
    return MCPT_OK;
}

int mcpt_num_monomers(mcpt_handle h) { return h ? (int)h->mons.size() : 0; }
int mcpt_num_dimers(mcpt_handle h) { return h ? (int)h->dims.size() : 0; }

const char* mcpt_last_error(mcpt_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void mcpt_destroy(mcpt_handle h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& P : h->plans) free_plan(h, P.get());
    for (void* p : h->owned) cudaFree(p);
    cudaFree(h->dC);
    cudaFree(h->dCf);
    cudaFree(h->dE);
    cudaFree(h->dH);
    cudaFree(h->dVT);
    cudaFree(h->dCoup);
    cudaFree(h->dR);
    cudaFree(h->dS1);
    cudaFree(h->dTd2);
    cudaFree(h->dTd2Tab);
    cudaFree(h->dTd2Mon);
    cudaFree(h->dTd2Out);
    cudaFree(h->dDf);
    cudaFree(h->dDfOut);
    cudaFree(h->dDfLists);
    for (int b = 0; b < 2; b++) {
        cudaFree(h->dPack[b]);
        if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
        if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
        if (h->copy_stream[b]) cudaStreamDestroy(h->copy_stream[b]);
    }
    cudaFree(h->dE2);
    cudaFree(h->dMon);
    cudaFree(h->dLists);
    cudaFree(h->dFlag);
    for (cudaEvent_t e : h->rev.pool) cudaEventDestroy(e);
    for (auto& v : h->rev.pending)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
