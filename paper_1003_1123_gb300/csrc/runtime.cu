// Handles, errors, seeding kernels, state blobs and statistics finishing.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

// ------------------------------------------------------------------ errors
static thread_local char g_msg[1024] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_msg[0] = 0; }

// --------------------------------------------------------------- devices
static std::mutex g_dev_mu;
static std::vector<DevInfo> g_dev;

int dev_info(int device, DevInfo* out)
{
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if ((int)g_dev.size() <= device) g_dev.resize(device + 1);
    DevInfo& d = g_dev[device];
    if (d.sms == 0) {
        GB_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device));
        GB_CUDA(cudaDeviceGetAttribute(&d.max_threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor,
                                       device));
        int optin = 0;
        GB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
        d.smem_optin = (size_t)optin;
    }
    *out = d;
    return GBRNG_OK;
}

// Process-wide settings (set from any host thread, read at each launch).
static std::atomic<uint64_t> g_wait_ns{2000000000ull};
uint64_t wait_limit_ns() { return g_wait_ns.load(); }

static std::atomic<int64_t> g_stall_chunk{-1};
int64_t test_stall_chunk() { return g_stall_chunk.load(); }

int ensure_partials(Handle* h, int64_t count)
{
    if (count <= h->partials_cap) return GBRNG_OK;
    if (h->partials) cudaFree(h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (cudaMalloc(&h->partials, sizeof(double) * 4 * count) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "cannot allocate %lld reduction partials", (long long)count);
    }
    h->partials_cap = count;
    return GBRNG_OK;
}

int ensure_eacc(Handle* h, int64_t n)
{
    if (n <= h->eacc_cap) return GBRNG_OK;
    if (h->eacc) cudaFree(h->eacc);
    h->eacc = nullptr;
    h->eacc_cap = 0;
    if (cudaMalloc(&h->eacc, sizeof(float2) * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "cannot allocate %lld energy sums", (long long)n);
    }
    h->eacc_cap = n;
    return GBRNG_OK;
}

int ensure_adj(Handle* h, size_t bytes)
{
    if (bytes <= h->adj_bytes) return GBRNG_OK;
    if (h->adj) cudaFree(h->adj);
    h->adj = nullptr;
    h->adj_bytes = 0;
    if (cudaMalloc((void**)&h->adj, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "adjoint scratch of %zu bytes", bytes);
    }
    h->adj_bytes = bytes;
    return GBRNG_OK;
}

int ensure_progress(Handle* h, int64_t count)
{
    if (count <= h->progress_cap) return GBRNG_OK;
    if (h->progress) cudaFree(h->progress);
    h->progress = nullptr;
    h->progress_cap = 0;
    if (cudaMalloc(&h->progress, sizeof(uint64_t) * count) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "cannot allocate %lld progress counters", (long long)count);
    }
    h->progress_cap = count;
    return GBRNG_OK;
}

// ------------------------------------------------------------ Table I
// (sl, ll) of Table I; row 4 prints sl = 12470, whose trinomial is
// reducible, and is used as 13470.
static const int32_t kLags[10][2] = {
    {1252, 2281},     {3004, 4423},     {5502, 9689},     {10095, 19937},
    {13470, 23209},   {23463, 44497},   {54454, 132049},  {279695, 756839},
    {288477, 859433}, {1010202, 3021377}};

int lfg_lags(int row, int32_t* sl, int32_t* ll)
{
    if (row < 0 || row > 9) return fail(GBRNG_ELAGS, "Table I has rows 0-9, got %d", row);
    if (sl) *sl = kLags[row][0];
    if (ll) *ll = kLags[row][1];
    return GBRNG_OK;
}

int lfg_default_row(int64_t n_threads)
{
    for (int r = 0; r < 10; ++r)
        if (kLags[r][0] > 4 * n_threads && kLags[r][1] - kLags[r][0] > 4 * n_threads) return r;
    return 9;
}

// ---------------------------------------------------------- seeding kernels
__global__ void taus_seed_kernel(uint64_t seed, int64_t n, uint4* st)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = (uint32_t)splitmix64_at(seed, 8ull * (uint64_t)s + k);
    if (w[0] < 2u) w[0] += 2u;
    if (w[1] < 8u) w[1] += 8u;
    if (w[2] < 16u) w[2] += 16u;
    st[s] = make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void lcg_seed_kernel(uint64_t seed, int64_t n, uint32_t* st)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) st[s] = (uint32_t)splitmix64_at(seed, 8ull * (uint64_t)s);
}

// Seeding part of Algorithm 2, per stream: idum2 <- idum, NTAB+8 Schrage steps,
// the last NTAB fill iv[]; iy starts as iv[0].  Layout [35][n].
__global__ void ran2_seed_kernel(uint64_t seed, int64_t n, int32_t* st)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint64_t w = splitmix64_at(seed, 8ull * (uint64_t)s);
    int32_t idum = 1 + (int32_t)(w % (uint64_t)kR2Imm1);
    st[1 * n + s] = idum;
    int32_t iv0 = 0;
    for (int j = 32 + 7; j >= 0; --j) {
        idum = schrage<kR2A1, kR2M1, kR2Q1, kR2R1>(idum);
        if (j < 32) st[(3 + j) * n + s] = idum;
        if (j == 0) iv0 = idum;
    }
    st[0 * n + s] = idum;
    st[2 * n + s] = iv0;
}

static int launch_seed(Handle* h, cudaStream_t st)
{
    const int T = 256;
    const int64_t blocks = (h->n + T - 1) / T;
    if (h->kind == GBRNG_TAUS)
        taus_seed_kernel<<<(unsigned)blocks, T, 0, st>>>(h->seed, h->n, h->taus);
    else if (h->kind == GBRNG_RAN2)
        ran2_seed_kernel<<<(unsigned)blocks, T, 0, st>>>(h->seed, h->n, h->r2);
    else if (h->kind == GBRNG_LCG)
        lcg_seed_kernel<<<(unsigned)blocks, T, 0, st>>>(h->seed, h->n, h->lcg);
    else
        return lfg_seed(h, st);
    GB_CUDA(cudaGetLastError());
    return GBRNG_OK;
}

static void free_handle(Handle* h)
{
    if (!h) return;
    cudaFree(h->taus);
    cudaFree(h->r2);
    cudaFree(h->lcg);
    cudaFree(h->ring);
    cudaFree(h->progress);
    cudaFree(h->dstatus);
    cudaFree(h->partials);
    cudaFree(h->dstats);
    cudaFree(h->eacc);
    cudaFree(h->adj);
    delete static_cast<gbrng_rng*>(h);
}

static int alloc_state(Handle* h)
{
    cudaError_t e = cudaSuccess;
    if (h->kind == GBRNG_TAUS) {
        e = cudaMalloc(&h->taus, sizeof(uint4) * h->n);
    } else if (h->kind == GBRNG_RAN2) {
        e = cudaMalloc(&h->r2, sizeof(int32_t) * 35 * h->n);
    } else if (h->kind == GBRNG_LCG) {
        e = cudaMalloc(&h->lcg, sizeof(uint32_t) * h->n);
    } else {
        // ring size: k (ll + D) rounded up to 32 words for the highest leap
        // order k the ring serves (2 unless order 4 was set before creation).
        // The order-k leap reads back to p - k ll, and a round of W <= k D
        // positions overwrites positions p - R, so R - k ll >= k D lets every
        // round take its full width (the seeds' backward extension fills
        // positions -k ll .. -1).
        h->order_max = lfg_order_for_new_handle();
        const uint64_t D = (uint64_t)(h->ll - h->sl);
        const uint64_t R = ((uint64_t)h->order_max * ((uint64_t)h->ll + D) + 31) & ~(uint64_t)31;
        h->ring_size = (uint32_t)R;
        e = cudaMalloc(&h->ring, sizeof(uint32_t) * (R + ring_mirror(h->ring_size)));
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->dstatus, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->dstats, sizeof(double) * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "cannot allocate generator state for %lld streams: %s",
                    (long long)h->n, cudaGetErrorString(e));
    }
    GB_CUDA(cudaMemset(h->dstatus, 0, sizeof(int)));
    return GBRNG_OK;
}

static int create(gbrng_t* out, int kind, uint64_t seed, int64_t n, int row, cudaStream_t st)
{
    if (!out) return fail(GBRNG_EINVAL, "out is NULL");
    *out = nullptr;
    if (kind < GBRNG_TAUS || kind > GBRNG_LCG) return fail(GBRNG_EINVAL, "unknown kind %d", kind);
    if (n < 1) return fail(GBRNG_EINVAL, "n_streams must be >= 1, got %lld", (long long)n);
    if (kind != GBRNG_LAGFIB && n > (int64_t)INT32_MAX * 16)
        return fail(GBRNG_EINVAL, "too many streams");
    gbrng_rng* h = new (std::nothrow) gbrng_rng();
    if (!h) return fail(GBRNG_ENOMEM, "host allocation failed");
    h->kind = kind;
    h->seed = seed;
    h->n = n;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(GBRNG_ECUDA, "no CUDA device");
    }
    if (kind == GBRNG_LAGFIB) {
        h->row = row < 0 ? lfg_default_row(n) : row;
        int rc = lfg_lags(h->row, &h->sl, &h->ll);
        if (rc != GBRNG_OK) {
            delete h;
            return rc;
        }
    }
    int rc = alloc_state(h);
    if (rc == GBRNG_OK) rc = launch_seed(h, st);
    if (rc != GBRNG_OK) {
        free_handle(h);
        return rc;
    }
    *out = h;
    return GBRNG_OK;
}

// ---------------------------------------------------------- statistics
// One block reduces `blocks` partials (4 doubles each, block-major) in a
// fixed order and writes sum_x2, sum_v2, sum_xv, energy sum.
__global__ void finish_stats_kernel(const double* partials, int64_t blocks, double* out)
{
    __shared__ double sm[4 * 32];
    double v[4] = {0, 0, 0, 0};
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partials[4 * b + k];
    block_reduce_sum<4>(v, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = v[k];
}

int finish_stats(Handle* h, int64_t blocks, int64_t n_steps, ld_stats* out, cudaStream_t st)
{
    if (!out) return GBRNG_OK;
    finish_stats_kernel<<<1, 256, 0, st>>>(h->partials, blocks, h->dstats);
    GB_CUDA(cudaGetLastError());
    double host[4];
    GB_CUDA(cudaMemcpyAsync(host, h->dstats, sizeof host, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    out->sum_x2 = host[0];
    out->sum_v2 = host[1];
    out->sum_xv = host[2];
    out->energy_time_avg = n_steps > 0 ? host[3] / (double)n_steps : 0.0;
    out->steps = n_steps;
    return GBRNG_OK;
}

// ------------------------------------------------------- systems
LdCoef make_coef(const ld_system* s)
{
    LdCoef c;
    c.cdt = (float)s->dt;
    c.cva = (float)(1.0 - (s->gamma * s->dt) / s->m);
    c.ckm = (float)(s->dt / s->m);
    c.cs = (float)(sqrt(2.0 * s->gamma * s->kT * s->dt) / s->m);
    c.sv = (float)sqrt(s->kT / s->m);
    c.kT = (float)s->kT;
    c.K = (float)s->K;
    c.hm = (float)(0.5 * s->m);
    return c;
}

int check_system(const ld_system* s, bool need_rng)
{
    if (!s) return fail(GBRNG_EINVAL, "system is NULL");
    if (s->n < 0) return fail(GBRNG_EINVAL, "n must be >= 0");
    if (s->n > 0 && (!s->x || !s->v)) return fail(GBRNG_EINVAL, "x and v must be device arrays");
    if (!(s->m > 0) || !(s->dt > 0) || !(s->gamma >= 0) || !(s->kT >= 0))
        return fail(GBRNG_EINVAL, "need m > 0, dt > 0, gamma >= 0, kT >= 0");
    if (!s->K_per && !(s->K > 0)) return fail(GBRNG_EINVAL, "need K > 0 or K_per");
    if (need_rng) {
        if (!s->rng) return fail(GBRNG_EINVAL, "system has no generator");
        if (s->rng->kind != GBRNG_LAGFIB && s->rng->n < s->n)
            return fail(GBRNG_EINVAL, "generator has %lld streams for %lld oscillators",
                        (long long)s->rng->n, (long long)s->n);
    }
    return GBRNG_OK;
}

}  // namespace gb

using namespace gb;

// ===================================================================== C ABI
extern "C" {

const char* gbrng_last_error(void) { return g_msg; }

int rng_set_wait_limit_ns(uint64_t ns)
{
    if (ns == 0) return fail(GBRNG_EINVAL, "wait limit must be > 0");
    g_wait_ns.store(ns);
    return GBRNG_OK;
}

int gbrng_test_stall_chunk(int64_t chunk)
{
    if (chunk < -1) return fail(GBRNG_EINVAL, "chunk must be >= -1");
    g_stall_chunk.store(chunk);
    return GBRNG_OK;
}

int rng_lfg_lags(int row, int32_t* sl, int32_t* ll) { return lfg_lags(row, sl, ll); }

int rng_lfg_default_row(int64_t n_threads)
{
    if (n_threads < 1) return fail(GBRNG_EINVAL, "n_threads must be >= 1");
    return lfg_default_row(n_threads);
}

int rng_init(gbrng_t* out, int kind, uint64_t seed, int64_t n_streams, void* stream)
{
    NvtxRange range("rng_init");
    return create(out, kind, seed, n_streams, -1, (cudaStream_t)stream);
}

int rng_init_lfg(gbrng_t* out, uint64_t seed, int64_t n_threads, int lag_row, void* stream)
{
    NvtxRange range("rng_init_lfg");
    if (lag_row < -1 || lag_row > 9) {
        if (out) *out = nullptr;
        return fail(GBRNG_ELAGS, "lag_row must be -1 or 0-9, got %d", lag_row);
    }
    return create(out, GBRNG_LAGFIB, seed, n_threads, lag_row, (cudaStream_t)stream);
}

int rng_destroy(gbrng_t rng)
{
    if (!rng) return fail(GBRNG_EINVAL, "handle is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(rng->device);
    cudaError_t e = cudaDeviceSynchronize();
    free_handle(rng);
    cudaSetDevice(dev);
    if (e != cudaSuccess) return fail(GBRNG_ECUDA, "pending work failed: %s", cudaGetErrorString(e));
    return GBRNG_OK;
}

int rng_clone(gbrng_t src, gbrng_t* out, void* stream)
{
    if (!src || !out) return fail(GBRNG_EINVAL, "NULL argument");
    *out = nullptr;
    gbrng_rng* h = new (std::nothrow) gbrng_rng();
    if (!h) return fail(GBRNG_ENOMEM, "host allocation failed");
    h->kind = src->kind;
    h->seed = src->seed;
    h->n = src->n;
    h->device = src->device;
    h->row = src->row;
    h->sl = src->sl;
    h->ll = src->ll;
    h->pos = src->pos;
    int rc = alloc_state(h);
    if (rc != GBRNG_OK) {
        free_handle(h);
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (h->kind == GBRNG_TAUS)
        e = cudaMemcpyAsync(h->taus, src->taus, sizeof(uint4) * h->n, cudaMemcpyDeviceToDevice, st);
    else if (h->kind == GBRNG_RAN2)
        e = cudaMemcpyAsync(h->r2, src->r2, sizeof(int32_t) * 35 * h->n, cudaMemcpyDeviceToDevice,
                            st);
    else if (h->kind == GBRNG_LCG)
        e = cudaMemcpyAsync(h->lcg, src->lcg, sizeof(uint32_t) * h->n, cudaMemcpyDeviceToDevice, st);
    else
        e = cudaMemcpyAsync(h->ring, src->ring,
                            sizeof(uint32_t) * ((size_t)h->ring_size + ring_mirror(h->ring_size)),
                            cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        free_handle(h);
        return fail(GBRNG_ECUDA, "clone copy failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    return GBRNG_OK;
}

int rng_info(gbrng_t rng, int* kind, int64_t* n_streams, int* lag_row, int64_t* position)
{
    if (!rng) return fail(GBRNG_EINVAL, "handle is NULL");
    if (kind) *kind = rng->kind;
    if (n_streams) *n_streams = rng->n;
    if (lag_row) *lag_row = rng->row;
    if (position) *position = rng->pos;
    return GBRNG_OK;
}

static size_t payload_bytes(const Handle* h)
{
    if (h->kind == GBRNG_TAUS) return sizeof(uint32_t) * 4 * (size_t)h->n;
    if (h->kind == GBRNG_RAN2) return sizeof(int32_t) * 35 * (size_t)h->n;
    if (h->kind == GBRNG_LCG) return sizeof(uint32_t) * (size_t)h->n;
    return sizeof(uint32_t) * (size_t)h->ll;
}

int rng_state_bytes(gbrng_t rng, size_t* bytes)
{
    if (!rng || !bytes) return fail(GBRNG_EINVAL, "NULL argument");
    *bytes = sizeof(gbrng_state_header) + payload_bytes(rng);
    return GBRNG_OK;
}

int rng_get_state(gbrng_t rng, void* host, size_t bytes)
{
    NvtxRange range("rng_get_state");
    if (!rng || !host) return fail(GBRNG_EINVAL, "NULL argument");
    const size_t pb = payload_bytes(rng);
    if (bytes != sizeof(gbrng_state_header) + pb)
        return fail(GBRNG_EINVAL, "state blob must be %zu bytes", sizeof(gbrng_state_header) + pb);
    gbrng_state_header hd;
    hd.magic = 0x4E524247u;
    hd.version = 1;
    hd.kind = rng->kind;
    hd.lag_row = rng->row;
    hd.n_streams = rng->n;
    hd.position = rng->pos;
    hd.payload_bytes = pb;
    memcpy(host, &hd, sizeof hd);
    char* dst = (char*)host + sizeof hd;
    GB_CUDA(cudaDeviceSynchronize());
    if (rng->kind == GBRNG_TAUS) {
        GB_CUDA(cudaMemcpy(dst, rng->taus, pb, cudaMemcpyDeviceToHost));
    } else if (rng->kind == GBRNG_LCG) {
        GB_CUDA(cudaMemcpy(dst, rng->lcg, pb, cudaMemcpyDeviceToHost));
    } else if (rng->kind == GBRNG_RAN2) {
        // device layout [35][n] -> blob [n][35]
        std::vector<int32_t> tmp((size_t)35 * rng->n);
        GB_CUDA(cudaMemcpy(tmp.data(), rng->r2, pb, cudaMemcpyDeviceToHost));
        int32_t* o = (int32_t*)dst;
        for (int64_t s = 0; s < rng->n; ++s)
            for (int k = 0; k < 35; ++k) o[35 * s + k] = tmp[(size_t)k * rng->n + s];
    } else {
        const int64_t R = rng->ring_size;
        std::vector<uint32_t> ring(R);
        GB_CUDA(cudaMemcpy(ring.data(), rng->ring, sizeof(uint32_t) * R, cudaMemcpyDeviceToHost));
        uint32_t* o = (uint32_t*)dst;
        for (int64_t k = 0; k < rng->ll; ++k) {
            const int64_t r = (rng->pos - rng->ll + k) % R;
            o[k] = ring[r < 0 ? r + R : r];
        }
    }
    return GBRNG_OK;
}

int rng_set_state(gbrng_t rng, const void* host, size_t bytes)
{
    NvtxRange range("rng_set_state");
    if (!rng || !host) return fail(GBRNG_EINVAL, "NULL argument");
    const size_t pb = payload_bytes(rng);
    if (bytes != sizeof(gbrng_state_header) + pb)
        return fail(GBRNG_ESTATE, "state blob must be %zu bytes", sizeof(gbrng_state_header) + pb);
    gbrng_state_header hd;
    memcpy(&hd, host, sizeof hd);
    if (hd.magic != 0x4E524247u || hd.version != 1 || hd.kind != rng->kind ||
        hd.n_streams != rng->n || hd.payload_bytes != pb ||
        (rng->kind == GBRNG_LAGFIB && hd.lag_row != rng->row) || hd.position < 0)
        return fail(GBRNG_ESTATE, "state blob does not match this handle");
    const char* src = (const char*)host + sizeof hd;
    GB_CUDA(cudaDeviceSynchronize());
    if (rng->kind == GBRNG_TAUS) {
        GB_CUDA(cudaMemcpy(rng->taus, src, pb, cudaMemcpyHostToDevice));
    } else if (rng->kind == GBRNG_LCG) {
        GB_CUDA(cudaMemcpy(rng->lcg, src, pb, cudaMemcpyHostToDevice));
    } else if (rng->kind == GBRNG_RAN2) {
        std::vector<int32_t> tmp((size_t)35 * rng->n);
        const int32_t* in = (const int32_t*)src;
        for (int64_t s = 0; s < rng->n; ++s)
            for (int k = 0; k < 35; ++k) tmp[(size_t)k * rng->n + s] = in[35 * s + k];
        GB_CUDA(cudaMemcpy(rng->r2, tmp.data(), pb, cudaMemcpyHostToDevice));
    } else {
        // The blob holds x_{p-ll} .. x_{p-1}.  The leap forms of the recurrence
        // also read x_{p-k ll} .. x_{p-ll-1} (k = the ring's highest order);
        // they follow from the recurrence run backwards, x_q = x_{q+ll} -
        // x_{q+sl}, which keeps the recurrence true at every index the leaps use.
        const int64_t R = rng->ring_size;
        const int64_t ll = rng->ll, sl = rng->sl, p = hd.position, k = rng->order_max;
        std::vector<uint32_t> hist((size_t)k * ll);          // hist[j] = x_{p-k ll+j}
        const uint32_t* in = (const uint32_t*)src;
        for (int64_t i = 0; i < ll; ++i) hist[(k - 1) * ll + i] = in[i];
        for (int64_t j = (k - 1) * ll - 1; j >= 0; --j) hist[j] = hist[j + ll] - hist[j + sl];
        const int64_t M = ring_mirror(rng->ring_size);
        std::vector<uint32_t> ring(R + M, 0u);
        for (int64_t j = 0; j < k * ll; ++j) {
            int64_t r = (p - k * ll + j) % R;
            if (r < 0) r += R;
            ring[r] = hist[j];
            if (r < M) ring[r + R] = hist[j];
        }
        GB_CUDA(cudaMemcpy(rng->ring, ring.data(), sizeof(uint32_t) * (R + M),
                           cudaMemcpyHostToDevice));
        rng->pos = hd.position;
    }
    return GBRNG_OK;
}

int rng_fill_u32(gbrng_t rng, uint32_t* dst, int64_t n, void* stream)
{
    NvtxRange range("rng_fill_u32");
    if (!rng || (n > 0 && !dst) || n < 0) return fail(GBRNG_EINVAL, "bad fill arguments");
    if (n == 0) return GBRNG_OK;
    if (rng->kind == GBRNG_LAGFIB) return lfg_fill(rng, dst, n, 0, (cudaStream_t)stream);
    return fill_u32_pt(rng, dst, n, (cudaStream_t)stream);
}

int rng_fill_uniform(gbrng_t rng, float* dst, int64_t n, void* stream)
{
    NvtxRange range("rng_fill_uniform");
    if (!rng || (n > 0 && !dst) || n < 0) return fail(GBRNG_EINVAL, "bad fill arguments");
    if (n == 0) return GBRNG_OK;
    if (rng->kind == GBRNG_LAGFIB) return lfg_fill(rng, dst, n, 1, (cudaStream_t)stream);
    return fill_uniform_pt(rng, dst, n, (cudaStream_t)stream);
}

int rng_fill_normal(gbrng_t rng, float* dst, int64_t n, void* stream)
{
    NvtxRange range("rng_fill_normal");
    if (!rng || (n > 0 && !dst) || n < 0 || (n & 1))
        return fail(GBRNG_EINVAL, "bad fill arguments (n must be even)");
    if ((uintptr_t)dst & 7u) return fail(GBRNG_EINVAL, "normal fill needs an 8-byte aligned dst");
    if (n == 0) return GBRNG_OK;
    if (rng->kind == GBRNG_LAGFIB) return lfg_fill(rng, dst, n, 2, (cudaStream_t)stream);
    return fill_normal_pt(rng, dst, n, (cudaStream_t)stream);
}

int ld_init_equilibrium(ld_system* sys, void* stream)
{
    NvtxRange range("ld_init_equilibrium");
    GB_CHECK(check_system(sys, true));
    if (sys->n == 0) return GBRNG_OK;
    if (sys->rng->kind == GBRNG_LAGFIB) return lfg_ld(sys, 0, 1, nullptr, (cudaStream_t)stream);
    return ld_init_pt(sys, (cudaStream_t)stream);
}

int ld_run(ld_system* sys, int64_t n_steps, ld_stats* out, void* stream)
{
    NvtxRange range("ld_run");
    GB_CHECK(check_system(sys, true));
    if (n_steps < 0) return fail(GBRNG_EINVAL, "n_steps must be >= 0");
    if (sys->rng->kind == GBRNG_LAGFIB) return lfg_ld(sys, n_steps, 0, out, (cudaStream_t)stream);
    return ld_run_pt(sys, n_steps, out, (cudaStream_t)stream);
}

int ou_run(ou_system* sys, int64_t n_steps, int64_t every, double* mean, double* corr, void* stream)
{
    NvtxRange range("ou_run");
    if (!sys) return fail(GBRNG_EINVAL, "system is NULL");
    if (sys->n < 1 || !sys->R) return fail(GBRNG_EINVAL, "need n >= 1 and a device array R");
    if (n_steps < 0 || every < 1) return fail(GBRNG_EINVAL, "need n_steps >= 0 and every >= 1");
    if (!(sys->k_sp > 0) || !(sys->xi > 0) || !(sys->kT >= 0) || !(sys->dt > 0))
        return fail(GBRNG_EINVAL, "need k_sp > 0, xi > 0, kT >= 0, dt > 0");
    if ((mean == nullptr) != (corr == nullptr))
        return fail(GBRNG_EINVAL, "mean_host and corr_host are both given or both NULL");
    if (!sys->rng) return fail(GBRNG_EINVAL, "system has no generator");
    if (sys->rng->kind != GBRNG_LAGFIB && sys->rng->n < sys->n)
        return fail(GBRNG_EINVAL, "generator has %lld streams for %lld particles",
                    (long long)sys->rng->n, (long long)sys->n);
    if (sys->rng->kind == GBRNG_LAGFIB)
        return lfg_ou(sys, n_steps, every, mean, corr, (cudaStream_t)stream);
    return ou_run_pt(sys, n_steps, every, mean, corr, (cudaStream_t)stream);
}

int ld_run_stepwise(ld_system* sys, int64_t n_steps, ld_stats* out, void* stream)
{
    NvtxRange range("ld_run_stepwise");
    GB_CHECK(check_system(sys, true));
    if (n_steps < 0) return fail(GBRNG_EINVAL, "n_steps must be >= 0");
    if (sys->rng->kind == GBRNG_LAGFIB)
        return lfg_ld_stepwise(sys, n_steps, out, (cudaStream_t)stream);
    return ld_run_stepwise_pt(sys, n_steps, out, (cudaStream_t)stream);
}

}  // extern "C"
