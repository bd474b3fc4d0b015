// api.cu -- the C ABI of libgbp: context, problem set-up (mesh validation and
// adjacency on the host, once per mesh), and the entry points of the hot path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gbp_internal.cuh"

using gbp::Control;

namespace {

gbp_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return GBP_OK;
    if (e == cudaErrorMemoryAllocation) return GBP_ERR_NO_MEMORY;
    return GBP_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(T **p, int64_t n)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n <= 0) n = 1;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)n);
}

template <class T>
void dfree(T **p)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void free_mesh_buffers(gbp_ctx *c)
{
    dfree(&c->xyz);
    dfree(&c->tets);
    dfree(&c->n2t_ptr);
    dfree(&c->n2t);
    dfree(&c->n2n_ptr);
    dfree(&c->n2n);
    dfree(&c->frec);
    dfree(&c->pc);
    dfree(&c->fib);
    dfree(&c->cf);
    dfree(&c->ct);
    dfree(&c->tf);
    dfree(&c->tv);
    dfree(&c->tlip);
    dfree(&c->phi);
    dfree(&c->rec);
    dfree(&c->chg);
    dfree(&c->stamp);
    dfree(&c->lists);
    dfree(&c->keys);
    dfree(&c->mu);
    dfree(&c->jac_x);
    dfree(&c->jac_acc);
    dfree(&c->jac_acc2);
    dfree(&c->adj_w);
    dfree(&c->adj_cand);
    dfree(&c->adj_pair);
    dfree(&c->adj_pairw);
    dfree(&c->adj_rec);
    dfree(&c->defer);
    dfree(&c->adj_done);
    dfree(&c->L);
    dfree(&c->Lbf);
    dfree(&c->Lscale);
    dfree(&c->Lrowsum);
    dfree(&c->on_idx);
    dfree(&c->on_bary);
    dfree(&c->on_t);
    c->site_cap = 0;
    c->site_b = 0;
    dfree(&c->dphi);
    dfree(&c->dx3);
    c->dx3_cap = 0;
    c->has_fib = c->has_vel = c->lip_valid = false;
    c->N = 0;
    c->K = 0;
    c->solve_gen = -1;
    c->rec_nb = 0;
}

gbp_status latched(gbp_ctx *c)
{
    // synchronise and read the device status word
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return from_cuda(e);
    e = cudaMemcpy(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost);
    if (e) return from_cuda(e);
    return (gbp_status)(c->h_ctl->status ? c->h_ctl->status : c->h_ctl->param_status);
}

__global__ void k_rowsum(int64_t n_v, const float *__restrict__ L, float *__restrict__ rowsum)
{
    __shared__ double red[32];
    const float *Ll = L + (int64_t)blockIdx.x * n_v;
    double acc = 0.0;
    for (int64_t n = threadIdx.x; n < n_v; n += blockDim.x) acc += (double)Ll[n];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) rowsum[blockIdx.x] = (float)v;
    }
}

// dst[r][q] = src[r][q] for q < sc, 0 beyond (rows of sc floats -> rows of dc)
__global__ void k_restride(int64_t rows, int sc, const float *__restrict__ src, int dc, float *__restrict__ dst)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= rows * dc) return;
    const int64_t r = g / dc;
    const int q = (int)(g - r * dc);
    dst[g] = q < sc ? src[r * sc + q] : 0.f;
}

cudaError_t restride(gbp_ctx *c, int64_t rows, int sc, const float *src, int dc, float *dst)
{
    const int64_t n = rows * dc;
    if (n <= 0) return cudaSuccess;
    k_restride<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(rows, sc, src, dc, dst);
    c->launches++;
    return cudaGetLastError();
}

bool valid_template(const gbp_template *t)
{
    return t && t->T >= 1 && t->T <= 4096 && t->tau > 0.f && std::isfinite(t->tau) && t->dt > 0.f &&
           std::isfinite(t->dt) && std::isfinite(t->t0) && std::isfinite(t->K0) && std::isfinite(t->K1);
}

}  // namespace

namespace gbp {
void flush_timing(gbp_ctx *c)
{
    if (c->ev_used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int p = 0; p + 1 < c->ev_used; p += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[p], c->ev_pool[p + 1]) == cudaSuccess) {
            c->ms[c->ev_cls[p / 2]] += ms;
            c->cls_launches[c->ev_cls[p / 2]] += 1;
        }
    }
    c->ev_used = 0;
}

void time_begin(gbp_ctx *c, int cls)
{
    if (!c->timing) return;
    if (c->ev_used + 2 > 64) flush_timing(c);
    c->ev_cls[c->ev_used / 2] = cls;
    cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
}

void time_end(gbp_ctx *c, int cls)
{
    (void)cls;
    if (!c->timing) return;
    cudaEventRecord(c->ev_pool[c->ev_used + 1], c->stream);
    c->ev_used += 2;
}
}  // namespace gbp

extern "C" {

const char *gbp_status_string(gbp_status s)
{
    switch (s) {
    case GBP_OK: return "ok";
    case GBP_ERR_INVALID_ARG: return "invalid argument";
    case GBP_ERR_BAD_MESH: return "bad mesh (inverted or degenerate tetrahedron, bad vertex id)";
    case GBP_ERR_NOT_SPD: return "conduction tensor not SPD (velocity <= 0 / not finite, zero fibre)";
    case GBP_ERR_NOT_CONVERGED: return "iteration limit reached";
    case GBP_ERR_TIMEOUT: return "bounded device wait ran out";
    case GBP_ERR_UNREACHABLE: return "vertices unreachable from the onsets";
    case GBP_ERR_CUDA: return "CUDA runtime error";
    case GBP_ERR_STATE: return "call order violated";
    case GBP_ERR_NO_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

gbp_status gbp_create(gbp_ctx **out, int device, void *stream)
{
    if (!out) return GBP_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(device);
    gbp_ctx *c = new gbp_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    cudaError_t e = cudaMalloc(&c->ctl, sizeof(Control));
    if (!e) e = cudaMemset(c->ctl, 0, sizeof(Control));
    if (!e) e = cudaMalloc(&c->bar_grp, sizeof(gbp::BarGroup) * gbp::GBP_BAR_GROUPS);
    if (!e) e = cudaMallocHost(&c->h_ctl, sizeof(Control));
    for (int i = 0; i < 64 && !e; ++i) e = cudaEventCreate(&c->ev_pool[i]);
    if (e || !coop) {
        gbp_destroy(c);
        return e ? from_cuda(e) : GBP_ERR_CUDA;
    }
    *out = c;
    return GBP_OK;
}

void gbp_destroy(gbp_ctx *c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_mesh_buffers(c);
    dfree(&c->ctl);
    dfree(&c->bar_grp);
    dfree(&c->ecg_part);
    dfree(&c->resid);
    dfree(&c->ecg_tmp);
    dfree(&c->dev_in);
    dfree(&c->dev_out);
    dfree(&c->bat_in);
    dfree(&c->bat_out);
    dfree(&c->loss_buf);
    dfree(&c->trace);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->pin_in) cudaFreeHost(c->pin_in);
    if (c->pin_out) cudaFreeHost(c->pin_out);
    for (int i = 0; i < 64; ++i)
        if (c->ev_pool[i]) cudaEventDestroy(c->ev_pool[i]);
    delete c;
}

gbp_status gbp_set_stream(gbp_ctx *c, void *stream)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)stream;
    return GBP_OK;
}

gbp_status gbp_synchronize(gbp_ctx *c)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return latched(c);
}

static gbp_status build_mesh(gbp_ctx *c, const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t,
                             int64_t n_real, int dim);
static cudaError_t ensure_batch(gbp_ctx *c, int B);

// Host validation of a tet mesh: sizes within the limits, coordinates
// finite, vertex ids in range and distinct within a tet, signed volume above
// 1e-15 diag^3 (right-handed, not degenerate).
static gbp_status check_tets(const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t)
{
    if (!xyz || !tets || n_v < 4 || n_t < 1 || n_v >= (1ll << 30) || n_t >= (1ll << 29))
        return GBP_ERR_INVALID_ARG;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < n_v; ++i)
        for (int r = 0; r < 3; ++r) {
            double v = xyz[3 * i + r];
            if (!std::isfinite(v)) return GBP_ERR_BAD_MESH;
            lo[r] = std::min(lo[r], v);
            hi[r] = std::max(hi[r], v);
        }
    double diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                            (hi[2] - lo[2]) * (hi[2] - lo[2]));
    double vtol = 1e-15 * diag * diag * diag;
    for (int64_t j = 0; j < n_t; ++j) {
        const int32_t *t = tets + 4 * j;
        for (int q = 0; q < 4; ++q)
            if (t[q] < 0 || t[q] >= n_v) return GBP_ERR_BAD_MESH;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (t[a] == t[b]) return GBP_ERR_BAD_MESH;
        double e[3][3];
        for (int a = 0; a < 3; ++a)
            for (int r = 0; r < 3; ++r) e[a][r] = (double)xyz[3 * t[a + 1] + r] - (double)xyz[3 * t[0] + r];
        double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (!(det / 6.0 > vtol)) return GBP_ERR_BAD_MESH;
    }
    return GBP_OK;
}

// Host validation of a triangle mesh: sizes within the limits, coordinates
// finite, ids in range and distinct, area above 1e-12 ext^2 counter-clockwise.
// lo / hi receive the bounding box.
static gbp_status check_tris(const float *xy, int64_t n_v, const int32_t *tris, int64_t n_t, double lo[2],
                             double hi[2])
{
    if (!xy || !tris || n_v < 3 || n_t < 1 || n_v + 1 >= (1ll << 30) || n_t >= (1ll << 29))
        return GBP_ERR_INVALID_ARG;
    lo[0] = lo[1] = 1e300;
    hi[0] = hi[1] = -1e300;
    for (int64_t i = 0; i < n_v; ++i)
        for (int r = 0; r < 2; ++r) {
            double v = xy[2 * i + r];
            if (!std::isfinite(v)) return GBP_ERR_BAD_MESH;
            lo[r] = std::min(lo[r], v);
            hi[r] = std::max(hi[r], v);
        }
    const double ext = std::max(hi[0] - lo[0], hi[1] - lo[1]);
    const double atol = 1e-12 * ext * ext;
    for (int64_t j = 0; j < n_t; ++j) {
        const int32_t *t = tris + 3 * j;
        for (int q = 0; q < 3; ++q)
            if (t[q] < 0 || t[q] >= n_v) return GBP_ERR_BAD_MESH;
        if (t[0] == t[1] || t[0] == t[2] || t[1] == t[2]) return GBP_ERR_BAD_MESH;
        const double ax = (double)xy[2 * t[1]] - xy[2 * t[0]], ay = (double)xy[2 * t[1] + 1] - xy[2 * t[0] + 1];
        const double bx = (double)xy[2 * t[2]] - xy[2 * t[0]], by = (double)xy[2 * t[2] + 1] - xy[2 * t[0] + 1];
        if (!(0.5 * (ax * by - ay * bx) > atol)) return GBP_ERR_BAD_MESH;  // counter-clockwise, not degenerate
    }
    return GBP_OK;
}

gbp_status gbp_check_mesh(const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t)
{
    return check_tets(xyz, n_v, tets, n_t);
}

gbp_status gbp_check_mesh_2d(const float *xy, int64_t n_v, const int32_t *tris, int64_t n_t)
{
    double lo[2], hi[2];
    return check_tris(xy, n_v, tris, n_t, lo, hi);
}

gbp_status gbp_upload_mesh(gbp_ctx *c, const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    const gbp_status st = check_tets(xyz, n_v, tets, n_t);
    if (st != GBP_OK) return st;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    return build_mesh(c, xyz, n_v, tets, n_t, n_v, 3);
}

// Host adjacency of a validated tet mesh.  Vertices from n_real on (the
// apex of a lifted triangle mesh) get an empty vertex->tet row and appear in
// no vertex->vertex row: they are never solved nor activated.
struct HostAdjacency {
    std::vector<int> n2t_ptr, n2t;  // vertex -> tet*4 + slot, rows in ascending code
    std::vector<int> n2n_ptr, n2n;  // vertex -> neighbours through a shared tet, sorted, unique
    std::vector<int4> frec;         // per n2t entry: the tet's other three vertices (slot order), code
    int max_deg = 0, max_nbr = 0;
};

static void build_adjacency(const int32_t *tets, int64_t n_v, int64_t n_t, int64_t n_real, HostAdjacency &h)
{
    h.n2t_ptr.assign(n_v + 1, 0);
    for (int64_t j = 0; j < n_t; ++j)
        for (int q = 0; q < 4; ++q)
            if (tets[4 * j + q] < n_real) h.n2t_ptr[tets[4 * j + q] + 1]++;
    for (int64_t i = 0; i < n_v; ++i) h.n2t_ptr[i + 1] += h.n2t_ptr[i];
    const int64_t n_faces = h.n2t_ptr[n_v];
    h.n2t.assign(n_faces, 0);
    {
        std::vector<int> cur(h.n2t_ptr.begin(), h.n2t_ptr.end() - 1);
        for (int64_t j = 0; j < n_t; ++j)
            for (int q = 0; q < 4; ++q)
                if (tets[4 * j + q] < n_real) h.n2t[cur[tets[4 * j + q]]++] = (int)(4 * j + q);
    }
    h.max_deg = h.max_nbr = 0;
    h.n2n_ptr.assign(n_v + 1, 0);
    h.n2n.clear();
    h.n2n.reserve((size_t)n_t * 3);
    std::vector<int> buf;
    for (int64_t i = 0; i < n_v; ++i) {
        int b = h.n2t_ptr[i], e = h.n2t_ptr[i + 1];
        h.max_deg = std::max(h.max_deg, e - b);
        buf.clear();
        for (int p = b; p < e; ++p) {
            int j = h.n2t[p] >> 2;
            for (int q = 0; q < 4; ++q) {
                int v = tets[4 * (int64_t)j + q];
                if (v != i && v < n_real) buf.push_back(v);
            }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        h.n2n.insert(h.n2n.end(), buf.begin(), buf.end());
        h.max_nbr = std::max(h.max_nbr, (int)buf.size());
        h.n2n_ptr[i + 1] = (int)h.n2n.size();
    }
    // face records in vertex->tet order: the three other vertices in slot order, code
    h.frec.resize(n_faces);
    for (int64_t e = 0; e < n_faces; ++e) {
        const int code = h.n2t[e];
        const int64_t j = code >> 2;
        const int s = code & 3;
        int f[3], q3 = 0;
        for (int q = 0; q < 4; ++q)
            if (q != s) f[q3++] = tets[4 * j + q];
        h.frec[e] = make_int4(f[0], f[1], f[2], code);
    }
}

gbp_status gbp_mesh_adjacency(const int32_t *tets, int64_t n_v, int64_t n_t, int64_t *n_faces, int64_t *n_nbr,
                              int32_t *n2t_ptr, int32_t *n2t, int32_t *n2n_ptr, int32_t *n2n, int32_t *frec)
{
    if (!tets || !n_faces || !n_nbr || n_v < 1 || n_t < 1 || n_v >= (1ll << 30) || n_t >= (1ll << 29))
        return GBP_ERR_INVALID_ARG;
    for (int64_t k = 0; k < 4 * n_t; ++k)
        if (tets[k] < 0 || tets[k] >= n_v) return GBP_ERR_BAD_MESH;
    HostAdjacency h;
    build_adjacency(tets, n_v, n_t, n_v, h);
    *n_faces = (int64_t)h.n2t.size();
    *n_nbr = (int64_t)h.n2n.size();
    if (!n2t_ptr || !n2t || !n2n_ptr || !n2n || !frec) return GBP_OK;  // sizes only
    std::copy(h.n2t_ptr.begin(), h.n2t_ptr.end(), n2t_ptr);
    std::copy(h.n2t.begin(), h.n2t.end(), n2t);
    std::copy(h.n2n_ptr.begin(), h.n2n_ptr.end(), n2n_ptr);
    std::copy(h.n2n.begin(), h.n2n.end(), n2n);
    for (size_t e = 0; e < h.frec.size(); ++e) {
        frec[4 * e] = h.frec[e].x;
        frec[4 * e + 1] = h.frec[e].y;
        frec[4 * e + 2] = h.frec[e].z;
        frec[4 * e + 3] = h.frec[e].w;
    }
    return GBP_OK;
}

// Adjacency, face records and device buffers of a validated tet mesh
// (n_real as in build_adjacency).
static gbp_status build_mesh(gbp_ctx *c, const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t,
                             int64_t n_real, int dim)
{
    HostAdjacency h;
    build_adjacency(tets, n_v, n_t, n_real, h);
    const int64_t n_faces = (int64_t)h.n2t.size();
    free_mesh_buffers(c);
    c->n_v = n_v;
    c->n_t = n_t;
    c->n_e = n_real;
    c->dim = dim;
    c->max_deg = h.max_deg;
    c->max_nbr = h.max_nbr;
    std::vector<float4> x4(n_v);
    for (int64_t i = 0; i < n_v; ++i) x4[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
    cudaError_t err = cudaSuccess;
#define CK(x)                                \
    do {                                     \
        if (!err) err = (x);                 \
    } while (0)
    CK(dalloc(&c->xyz, n_v));
    CK(dalloc(&c->tets, n_t));
    CK(dalloc(&c->n2t_ptr, n_v + 1));
    CK(dalloc(&c->n2t, n_faces));
    CK(dalloc(&c->n2n_ptr, n_v + 1));
    CK(dalloc(&c->n2n, (int64_t)h.n2n.size()));
    CK(dalloc(&c->frec, n_faces));
    CK(dalloc(&c->pc, n_v));
    CK(dalloc(&c->fib, 3 * n_t));
    CK(dalloc(&c->cf, n_t));
    CK(dalloc(&c->ct, n_t));
    CK(dalloc(&c->tf, n_t));
    CK(dalloc(&c->tv, n_t));
    CK(dalloc(&c->tlip, n_t));
    CK(dalloc(&c->phi, n_v));
    CK(dalloc(&c->rec, n_v));
    CK(dalloc(&c->chg, n_v));
    CK(dalloc(&c->stamp, n_v));
    CK(dalloc(&c->lists, 4 * n_v + 32));
    CK(dalloc(&c->keys, n_v));
    CK(dalloc(&c->mu, n_v));
    CK(dalloc(&c->jac_x, n_v));
    CK(dalloc(&c->jac_acc, n_v));
    CK(dalloc(&c->jac_acc2, n_v));
    CK(dalloc(&c->adj_w, n_v));
    CK(dalloc(&c->adj_cand, n_v));
    CK(dalloc(&c->adj_pair, n_v));
    CK(dalloc(&c->adj_pairw, n_v));
    CK(dalloc(&c->adj_rec, 2 * n_v));
    CK(dalloc(&c->defer, gbp::FIM_DEFER_CAP));
    CK(dalloc(&c->adj_done, (n_v + 31) / 32 + 1));
    CK(dalloc(&c->dphi, n_v));
    CK(cudaMemset(c->dphi, 0, sizeof(float) * n_v));
    CK(cudaMemcpy(c->xyz, x4.data(), sizeof(float4) * n_v, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->tets, tets, sizeof(int4) * n_t, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->n2t_ptr, h.n2t_ptr.data(), sizeof(int) * (n_v + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->n2t, h.n2t.data(), sizeof(int) * n_faces, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->n2n_ptr, h.n2n_ptr.data(), sizeof(int) * (n_v + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->n2n, h.n2n.data(), sizeof(int) * h.n2n.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->frec, h.frec.data(), sizeof(int4) * h.frec.size(), cudaMemcpyHostToDevice));
#undef CK
    if (err) {
        free_mesh_buffers(c);
        c->n_v = c->n_t = c->n_e = 0;
        return from_cuda(err);
    }
    c->nb = 1;
    c->nb_cap = 1;
    c->param_gen++;
    return GBP_OK;
}

gbp_status gbp_upload_mesh_2d(gbp_ctx *c, const float *xy, int64_t n_v, const int32_t *tris, int64_t n_t)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    double lo[2], hi[2];
    const gbp_status st = check_tris(xy, n_v, tris, n_t, lo, hi);
    if (st != GBP_OK) return st;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    const double ext = std::max(hi[0] - lo[0], hi[1] - lo[1]);
    // lift: (x, y, 0) and the apex above the centre of the bounding box; any
    // height works (the apex is never reached), the extent keeps the tets well shaped
    std::vector<float> xyz(3 * (n_v + 1));
    for (int64_t i = 0; i < n_v; ++i) {
        xyz[3 * i] = xy[2 * i];
        xyz[3 * i + 1] = xy[2 * i + 1];
        xyz[3 * i + 2] = 0.f;
    }
    xyz[3 * n_v] = (float)(0.5 * (lo[0] + hi[0]));
    xyz[3 * n_v + 1] = (float)(0.5 * (lo[1] + hi[1]));
    xyz[3 * n_v + 2] = (float)(ext > 0 ? ext : 1.0);
    std::vector<int32_t> tets(4 * n_t);
    for (int64_t j = 0; j < n_t; ++j) {
        for (int q = 0; q < 3; ++q) tets[4 * j + q] = tris[3 * j + q];
        tets[4 * j + 3] = (int32_t)n_v;
    }
    return build_mesh(c, xyz.data(), n_v + 1, tets.data(), n_t, n_v, 2);
}

gbp_status gbp_set_fibres(gbp_ctx *c, const float *fib)
{
    if (!c || !fib) return GBP_ERR_INVALID_ARG;
    if (!c->n_t) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    cudaError_t e = c->dim == 2 ? restride(c, c->n_t, 2, fib, 3, c->fib)
                                : cudaMemcpyAsync(c->fib, fib, sizeof(float) * 3 * c->n_t, cudaMemcpyDeviceToDevice,
                                                  c->stream);
    if (e) return from_cuda(e);
    c->has_fib = true;
    c->has_vel = false;
    c->lip_valid = false;
    c->param_gen++;
    return GBP_OK;
}

gbp_status gbp_set_velocities(gbp_ctx *c, const float *cf, const float *ct)
{
    if (!c || !cf || !ct) return GBP_ERR_INVALID_ARG;
    if (!c->n_t || !c->has_fib) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    c->nb = 1;  // one problem from here on
    cudaError_t e = cudaSuccess;
    if (cf != c->cf) e = cudaMemcpyAsync(c->cf, cf, sizeof(float) * c->n_t, cudaMemcpyDeviceToDevice, c->stream);
    if (!e && ct != c->ct)
        e = cudaMemcpyAsync(c->ct, ct, sizeof(float) * c->n_t, cudaMemcpyDeviceToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(&c->ctl->param_status, 0, sizeof(int), c->stream);
    if (!e) {
        gbp::time_begin(c, 5);
        e = gbp::launch_precompute(c);
        gbp::time_end(c, 5);
    }
    if (e) return from_cuda(e);
    c->has_vel = true;
    c->lip_valid = false;
    c->param_gen++;
    return GBP_OK;
}

gbp_status gbp_set_leadfield(gbp_ctx *c, const float *L, int32_t N)
{
    if (!c || !L || N < 1 || N > 16) return GBP_ERR_INVALID_ARG;
    if (!c->n_v) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    cudaError_t e = dalloc(&c->L, (int64_t)N * c->n_e);
    if (!e) e = dalloc(&c->Lrowsum, 16);
    if (!e) e = cudaMemcpyAsync(c->L, L, sizeof(float) * N * c->n_e, cudaMemcpyDeviceToDevice, c->stream);
    if (!e) {
        k_rowsum<<<N, 256, 0, c->stream>>>(c->n_e, c->L, c->Lrowsum);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e) return from_cuda(e);
    c->N = N;
    e = gbp::prepare_leadfield_bf16(c);
    return from_cuda(e);
}

// Copy n site entries (ids, barycentric coordinates in the caller's layout,
// times) into the context's onset arrays, growing them first.  on_t keeps
// room for K times per problem of the batch capacity.
static cudaError_t store_sites(gbp_ctx *c, int32_t kind, int32_t K, int64_t n, const int32_t *idx, const float *bary,
                               const float *t)
{
    cudaError_t e = cudaSuccess;
    if (n > c->site_cap) {
        e = dalloc(&c->on_idx, n);
        if (!e) e = dalloc(&c->on_bary, 4 * n);
        c->site_cap = e ? 0 : n;
    }
    const int64_t nt = std::max<int64_t>(n, (int64_t)K * c->nb_cap);
    if (!e && (K != c->K || n > (int64_t)K * c->nb_cap)) e = dalloc(&c->on_t, nt);
    if (!e) e = cudaMemcpyAsync(c->on_idx, idx, sizeof(int) * n, cudaMemcpyDeviceToDevice, c->stream);
    if (!e && kind == GBP_ONSET_ELEMENT)
        e = c->dim == 2 ? restride(c, n, 3, bary, 4, c->on_bary)
                        : cudaMemcpyAsync(c->on_bary, bary, sizeof(float) * 4 * n, cudaMemcpyDeviceToDevice,
                                          c->stream);
    if (!e && kind == GBP_ONSET_NODAL) e = cudaMemsetAsync(c->on_bary, 0, sizeof(float) * 4 * n, c->stream);
    if (!e) e = cudaMemcpyAsync(c->on_t, t, sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream);
    return e;
}

gbp_status gbp_set_onsets(gbp_ctx *c, int32_t kind, int32_t K, const int32_t *idx, const float *bary,
                          const float *t)
{
    if (!c || !idx || !t || K < 1 || K > 65536) return GBP_ERR_INVALID_ARG;
    if (kind != GBP_ONSET_NODAL && kind != GBP_ONSET_ELEMENT) return GBP_ERR_INVALID_ARG;
    if (kind == GBP_ONSET_ELEMENT && !bary) return GBP_ERR_INVALID_ARG;
    if (!c->n_v) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    cudaError_t e = store_sites(c, kind, K, K, idx, bary, t);
    if (e) return from_cuda(e);
    c->K = K;
    c->onset_kind = kind;
    c->site_b = 0;
    c->param_gen++;
    return GBP_OK;
}

gbp_status gbp_set_onsets_batch(gbp_ctx *c, int32_t kind, int32_t B, int32_t K, const int32_t *idx,
                                const float *bary, const float *t)
{
    if (!c || !idx || !t || B < 1 || K < 1 || K > 65536) return GBP_ERR_INVALID_ARG;
    if (kind != GBP_ONSET_NODAL && kind != GBP_ONSET_ELEMENT) return GBP_ERR_INVALID_ARG;
    if (kind == GBP_ONSET_ELEMENT && !bary) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || c->nb_cap < 1) return GBP_ERR_STATE;
    if ((int64_t)B * c->n_v >= (1ll << 31) / 3 || (int64_t)B * K >= (1ll << 31) / 4) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = ensure_batch(c, B);
    if (!e) e = store_sites(c, kind, K, (int64_t)B * K, idx, bary, t);
    if (e) return from_cuda(e);
    c->K = K;
    c->onset_kind = kind;
    c->site_b = B;
    c->param_gen++;
    return GBP_OK;
}

static gbp_solve_opts normalized_opts(const gbp_ctx *c, const gbp_solve_opts *o)
{
    gbp_solve_opts r;
    if (o) r = *o;
    else {
        r.local_solver = GBP_LOCAL_EXACT;
        r.n_f = 32;
        r.eps = 0.f;
        r.max_iters = 0;
    }
    if (r.max_iters <= 0)
        r.max_iters = (int)(8.0 * (c->dim == 2 ? std::sqrt((double)c->n_v) : std::cbrt((double)c->n_v))) + 64 + r.n_f;
    return r;
}

gbp_status gbp_eikonal_solve(gbp_ctx *c, const gbp_solve_opts *opts, float *phi, int32_t *parent, float *alpha)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || !c->has_vel || !c->K) return GBP_ERR_STATE;
    gbp_solve_opts o = normalized_opts(c, opts);
    if (o.local_solver != GBP_LOCAL_EXACT && o.local_solver != GBP_LOCAL_FISTA) return GBP_ERR_INVALID_ARG;
    if (o.local_solver == GBP_LOCAL_FISTA && (o.n_f < 1 || o.n_f > 256)) return GBP_ERR_INVALID_ARG;
    if (!(o.eps >= 0.f) || !std::isfinite(o.eps)) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaSuccess;
    if (o.local_solver == GBP_LOCAL_FISTA && !c->lip_valid) {
        gbp::time_begin(c, 5);
        e = gbp::launch_lipschitz(c);
        gbp::time_end(c, 5);
        if (e) return from_cuda(e);
        c->lip_valid = true;
    }
    // keep a NOT_SPD latched by the precompute: the solve resets the control block
    e = gbp::launch_fim(c, &o);
    if (!e) e = gbp::launch_parent_pass(c, o.local_solver, o.n_f, phi, parent, alpha);
    if (e) return from_cuda(e);
    c->last_mode = o.local_solver;
    c->last_nf = o.n_f;
    c->solve_gen = c->param_gen;
    c->rec_nb = 1;
    return GBP_OK;
}

gbp_status gbp_get_solve_stats(gbp_ctx *c, gbp_solve_stats *s)
{
    if (!c || !s) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    gbp_status st = latched(c);
    if (st == GBP_ERR_CUDA || st == GBP_ERR_NO_MEMORY) return st;
    const Control &h = *c->h_ctl;
    s->iterations = h.iterations;
    s->candidates = (int64_t)h.candidates;
    s->face_updates = (int64_t)h.face_updates;
    s->fp64_fallbacks = (int64_t)h.fp64_fallbacks;
    s->unreached = (int64_t)h.unreached;
    s->adj_levels = h.adj_levels;
    s->adj_cycle_nodes = h.adj_cycle_nodes;
    s->adj_cycle_iters = h.adj_cycle_iters;
    s->status = h.status ? h.status : h.param_status;
    s->reserved = 0;
    s->adj_dataflow_ms = h.adj_ts[1] > h.adj_ts[0] ? (double)(h.adj_ts[1] - h.adj_ts[0]) * 1e-6 : 0.0;
    s->adj_cycle_ms = h.adj_ts[2] > h.adj_ts[1] ? (double)(h.adj_ts[2] - h.adj_ts[1]) * 1e-6 : 0.0;
    s->fim_deferred = h.n_defer;
    s->fim_repaired = h.n_repaired;
    return (gbp_status)s->status;
}

gbp_status gbp_ecg_forward(gbp_ctx *c, const float *phi, const gbp_template *tmpl, int32_t precision, float *ecg)
{
    if (!c || !phi || !ecg || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (precision != GBP_PREC_FP32 && precision != GBP_PREC_BF16) return GBP_ERR_INVALID_ARG;
    if (!c->N) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    return from_cuda(gbp::launch_ecg_forward(c, phi, tmpl, precision, ecg));
}

gbp_status gbp_ecg_loss_backward(gbp_ctx *c, const float *phi, const float *ecg, const float *target,
                                 const gbp_template *tmpl, float *loss, float *dphi)
{
    if (!c || !phi || !ecg || !target || !loss || !dphi || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (!c->N) return GBP_ERR_STATE;
    if ((int64_t)c->N * tmpl->T > 51200) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return from_cuda(gbp::launch_ecg_backward(c, phi, ecg, target, tmpl, loss, dphi));
}

// The adjoint of the current solve (or batch of solves).  For a lifted
// triangle mesh the caller's dLoss/dphi (n_e entries) is first copied into
// the context's own array (the apex entries are never read: the apex is
// unreached), and the onset-position gradient, computed as [..][3] with a
// zero third component, is repacked to [..][2].
static cudaError_t run_adjoint(gbp_ctx *c, const float *dphi, float *d_cf, float *d_ct, float *d_t, float *d_x)
{
    if (c->dim != 2) return gbp::launch_adjoint(c, dphi, d_cf, d_ct, d_t, d_x);
    cudaError_t e = cudaSuccess;
    if (dphi != c->dphi) {
        e = cudaMemcpyAsync(c->dphi, dphi, sizeof(float) * c->n_e, cudaMemcpyDeviceToDevice, c->stream);
        dphi = c->dphi;
    }
    float *dx3 = nullptr;
    if (!e && d_x) {
        const int64_t need = 3 * (int64_t)c->K * c->nb;
        if (need > c->dx3_cap) {
            e = dalloc(&c->dx3, need);
            c->dx3_cap = e ? 0 : need;
        }
        dx3 = c->dx3;
    }
    if (!e) e = gbp::launch_adjoint(c, dphi, d_cf, d_ct, d_t, dx3);
    if (!e && d_x) e = restride(c, (int64_t)c->K * c->nb, 3, dx3, 2, d_x);
    return e;
}

gbp_status gbp_geodesic_backward(gbp_ctx *c, const float *dphi, float *d_cf, float *d_ct, float *d_t, float *d_x)
{
    if (!c || !dphi) return GBP_ERR_INVALID_ARG;
    if (c->solve_gen < 0 || c->solve_gen != c->param_gen) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    return from_cuda(run_adjoint(c, dphi, d_cf, d_ct, d_t, d_x));
}

gbp_status gbp_forward_backward(gbp_ctx *c, const gbp_solve_opts *opts, const gbp_template *tmpl,
                                int32_t precision, const float *cf, const float *ct, const float *t,
                                const float *target, float *loss, float *ecg, float *d_cf, float *d_ct,
                                float *d_t, float *d_x)
{
    if (!c || !cf || !ct || !target || !loss || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || !c->has_fib || !c->K || !c->N) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    gbp_status st = gbp_set_velocities(c, cf, ct);
    if (st) return st;
    if (t) {
        cudaError_t e = cudaMemcpyAsync(c->on_t, t, sizeof(float) * c->K, cudaMemcpyDeviceToDevice, c->stream);
        if (e) return from_cuda(e);
        c->param_gen++;
    }
    st = gbp_eikonal_solve(c, opts, nullptr, nullptr, nullptr);
    if (st) return st;
    int64_t NT = (int64_t)c->N * tmpl->T;
    float *V = ecg;
    if (!V) {
        if (NT > c->ecg_tmp_cap) {
            cudaError_t e = dalloc(&c->ecg_tmp, NT);
            if (e) return from_cuda(e);
            c->ecg_tmp_cap = NT;
        }
        V = c->ecg_tmp;
    }
    st = gbp_ecg_forward(c, c->phi, tmpl, precision, V);
    if (st) return st;
    st = gbp_ecg_loss_backward(c, c->phi, V, target, tmpl, loss, c->dphi);
    if (st) return st;
    return gbp_geodesic_backward(c, c->dphi, d_cf, d_ct, d_t, d_x);
}

gbp_status gbp_forward_backward_host(gbp_ctx *c, const gbp_solve_opts *opts, const gbp_template *tmpl,
                                     int32_t precision, const float *cf, const float *ct, const float *t,
                                     const float *target, float *loss, float *d_cf, float *d_ct, float *d_t,
                                     float *d_x)
{
    if (!c || !cf || !ct || !target || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || !c->has_fib || !c->K || !c->N) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    const int64_t n_t = c->n_t, K = c->K, NT = (int64_t)c->N * tmpl->T, d = c->dim;
    // staging layout: in = [cf | ct | t | target], out = [loss | d_cf | d_ct | d_t | d_x]
    const int64_t in_n = 2 * n_t + K + NT, out_n = 1 + 2 * n_t + (1 + d) * K;
    cudaError_t e = cudaSuccess;
    if (in_n > c->stage_in_cap) {
        if (c->pin_in) cudaFreeHost(c->pin_in);
        c->pin_in = nullptr;
        e = dalloc(&c->dev_in, in_n);
        if (!e) e = cudaMallocHost(&c->pin_in, sizeof(float) * in_n);
        if (e) return from_cuda(e);
        c->stage_in_cap = in_n;
    }
    if (out_n > c->stage_out_cap) {
        if (c->pin_out) cudaFreeHost(c->pin_out);
        c->pin_out = nullptr;
        e = dalloc(&c->dev_out, out_n);
        if (!e) e = cudaMallocHost(&c->pin_out, sizeof(float) * out_n);
        if (e) return from_cuda(e);
        c->stage_out_cap = out_n;
    }
    float *pi = c->pin_in, *po = c->pin_out, *di = c->dev_in, *dout = c->dev_out;
    std::memcpy(pi, cf, sizeof(float) * n_t);
    std::memcpy(pi + n_t, ct, sizeof(float) * n_t);
    if (t) std::memcpy(pi + 2 * n_t, t, sizeof(float) * K);
    std::memcpy(pi + 2 * n_t + K, target, sizeof(float) * NT);
    e = cudaMemcpyAsync(di, pi, sizeof(float) * in_n, cudaMemcpyHostToDevice, c->stream);
    if (e) return from_cuda(e);
    gbp_status st = gbp_forward_backward(c, opts, tmpl, precision, di, di + n_t, t ? di + 2 * n_t : nullptr,
                                         di + 2 * n_t + K, dout, nullptr, dout + 1, dout + 1 + n_t,
                                         dout + 1 + 2 * n_t, dout + 1 + 2 * n_t + K);
    if (st) return st;
    e = cudaMemcpyAsync(po, dout, sizeof(float) * out_n, cudaMemcpyDeviceToHost, c->stream);
    if (e) return from_cuda(e);
    st = latched(c);
    if (st) return st;
    if (loss) *loss = po[0];
    if (d_cf) std::memcpy(d_cf, po + 1, sizeof(float) * n_t);
    if (d_ct) std::memcpy(d_ct, po + 1 + n_t, sizeof(float) * n_t);
    if (d_t) std::memcpy(d_t, po + 1 + 2 * n_t, sizeof(float) * K);
    if (d_x) std::memcpy(d_x, po + 1 + 2 * n_t + K, sizeof(float) * d * K);
    return GBP_OK;
}

// Grow the per-problem arrays to hold B problems (contents are not kept,
// except the first K onset times).
static cudaError_t ensure_batch(gbp_ctx *c, int B)
{
    if (B > c->nb_cap) c->rec_nb = 0;  // the per-problem arrays are rebuilt
    if (B <= c->nb_cap) return cudaSuccess;
    const int64_t nv = c->n_v * B, nt = c->n_t * B;
    cudaError_t err = cudaSuccess;
#define CK(x)                                \
    do {                                     \
        if (!err) err = (x);                 \
    } while (0)
    CK(cudaStreamSynchronize(c->stream));
    CK(dalloc(&c->cf, nt));
    CK(dalloc(&c->ct, nt));
    CK(dalloc(&c->tv, nt));
    CK(dalloc(&c->tlip, nt));
    CK(dalloc(&c->phi, nv));
    CK(dalloc(&c->rec, nv));
    CK(dalloc(&c->chg, nv));
    CK(dalloc(&c->stamp, nv));
    CK(dalloc(&c->lists, 4 * nv + 32));
    CK(dalloc(&c->keys, nv));
    CK(dalloc(&c->mu, nv));
    CK(dalloc(&c->jac_x, nv));
    CK(dalloc(&c->jac_acc, nv));
    CK(dalloc(&c->jac_acc2, nv));
    CK(dalloc(&c->adj_w, nv));
    CK(dalloc(&c->adj_cand, nv));
    CK(dalloc(&c->adj_pair, nv));
    CK(dalloc(&c->adj_pairw, nv));
    CK(dalloc(&c->adj_rec, 2 * nv));
    CK(dalloc(&c->adj_done, (nv + 31) / 32 + 1));
    CK(dalloc(&c->dphi, nv));
    CK(dalloc(&c->pc, nv));
    if (c->K && !err) {
        // grow the onset times keeping problem 0's (the shared times of gbp_set_onsets)
        float *nt_ = nullptr;
        CK(dalloc(&nt_, (int64_t)c->K * B));
        CK(cudaMemcpy(nt_, c->on_t, sizeof(float) * c->K, cudaMemcpyDeviceToDevice));
        if (!err) {
            dfree(&c->on_t);
            c->on_t = nt_;
        } else {
            dfree(&nt_);
        }
    }
#undef CK
    c->has_vel = false;
    c->lip_valid = false;
    c->solve_gen = -1;
    c->param_gen++;
    if (err) {
        c->nb_cap = 0;  // every per-problem array must be rebuilt by a new mesh upload
        return err;
    }
    c->nb_cap = B;
    return cudaSuccess;
}

gbp_status gbp_forward_backward_batch(gbp_ctx *c, int32_t B, const gbp_solve_opts *opts, const gbp_template *tmpl,
                                      int32_t precision, const float *cf, const float *ct, const float *t,
                                      const float *target, float *loss, float *ecg, float *d_cf, float *d_ct,
                                      float *d_t, float *d_x)
{
    if (!c || B < 1 || !cf || !ct || !target || !loss || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (precision != GBP_PREC_FP32 && precision != GBP_PREC_BF16) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || !c->has_fib || !c->K || !c->N || c->nb_cap < 1) return GBP_ERR_STATE;
    if (c->site_b > 0 && B != c->site_b) return GBP_ERR_STATE;  // per-problem sites are for B problems
    if ((int64_t)B * c->n_v >= (1ll << 31) / 3 || (int64_t)B * c->n_t >= (1ll << 31)) return GBP_ERR_INVALID_ARG;
    if ((int64_t)c->N * tmpl->T > 51200) return GBP_ERR_INVALID_ARG;
    gbp_solve_opts o = normalized_opts(c, opts);
    if (o.local_solver != GBP_LOCAL_EXACT && o.local_solver != GBP_LOCAL_FISTA) return GBP_ERR_INVALID_ARG;
    if (o.local_solver == GBP_LOCAL_FISTA && (o.n_f < 1 || o.n_f > 256)) return GBP_ERR_INVALID_ARG;
    if (!(o.eps >= 0.f) || !std::isfinite(o.eps)) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = ensure_batch(c, B);
    if (e) return from_cuda(e);
    const int64_t n_v = c->n_v, n_t = c->n_t, K = c->K, NT = (int64_t)c->N * tmpl->T;
    float *V = ecg;
    if (!V) {
        if (NT * B > c->ecg_tmp_cap) {
            e = dalloc(&c->ecg_tmp, NT * B);
            if (e) return from_cuda(e);
            c->ecg_tmp_cap = NT * B;
        }
        V = c->ecg_tmp;
    }
    c->nb = B;
    e = cudaMemcpyAsync(c->cf, cf, sizeof(float) * n_t * B, cudaMemcpyDeviceToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(c->ct, ct, sizeof(float) * n_t * B, cudaMemcpyDeviceToDevice, c->stream);
    if (t) {
        if (!e) e = cudaMemcpyAsync(c->on_t, t, sizeof(float) * K * B, cudaMemcpyDeviceToDevice, c->stream);
    } else if (c->site_b == 0) {
        for (int b = 1; b < B && !e; ++b)
            e = cudaMemcpyAsync(c->on_t + b * K, c->on_t, sizeof(float) * K, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (!e) e = cudaMemsetAsync(&c->ctl->param_status, 0, sizeof(int), c->stream);
    if (!e) {
        gbp::time_begin(c, 5);
        e = gbp::launch_precompute(c);
        gbp::time_end(c, 5);
    }
    if (!e && o.local_solver == GBP_LOCAL_FISTA) {
        gbp::time_begin(c, 5);
        e = gbp::launch_lipschitz(c);
        gbp::time_end(c, 5);
    }
    if (!e) e = gbp::launch_fim(c, &o);
    if (!e) e = gbp::launch_parent_pass(c, o.local_solver, o.n_f, nullptr, nullptr, nullptr);
    c->rec_nb = e ? 0 : B;
    // the ECG and misfit of all B problems in one launch each (the BF16
    // forward still runs problem by problem)
    if (precision == GBP_PREC_BF16) {
        for (int b = 0; b < B && !e; ++b) e = gbp::launch_ecg_forward(c, c->phi + b * n_v, tmpl, precision, V + b * NT);
    } else if (!e) {
        e = gbp::launch_ecg_forward_fp32_batch(c, B, c->phi, n_v, tmpl, V);
    }
    if (!e) e = gbp::launch_ecg_backward_batch(c, B, c->phi, n_v, V, target, tmpl, loss, c->dphi);
    if (!e) e = run_adjoint(c, c->dphi, d_cf, d_ct, d_t, d_x);
    // the context's single-problem state is gone: the next single-problem
    // evaluation starts from gbp_set_velocities
    c->nb = 1;
    c->has_vel = false;
    c->lip_valid = false;
    c->solve_gen = -1;
    c->param_gen++;
    return from_cuda(e);
}

gbp_status gbp_forward_backward_batch_host(gbp_ctx *c, int32_t B, const gbp_solve_opts *opts,
                                           const gbp_template *tmpl, int32_t precision, const float *cf,
                                           const float *ct, const float *t, const float *target, float *loss,
                                           float *d_cf, float *d_ct, float *d_t, float *d_x)
{
    if (!c || B < 1 || !cf || !ct || !target || !valid_template(tmpl)) return GBP_ERR_INVALID_ARG;
    if (!c->n_v || !c->has_fib || !c->K || !c->N) return GBP_ERR_STATE;
    DeviceGuard g(c->device);
    const int64_t n_t = c->n_t, K = c->K, NT = (int64_t)c->N * tmpl->T, d = c->dim;
    // device staging: in = [cf | ct | t | target], out = [loss | d_cf | d_ct | d_t | d_x], each [B][..]
    const int64_t in_n = B * (2 * n_t + K + NT), out_n = B * (1 + 2 * n_t + (1 + d) * K);
    cudaError_t e = cudaSuccess;
    if (in_n > c->bat_in_cap) {
        e = dalloc(&c->bat_in, in_n);
        c->bat_in_cap = e ? 0 : in_n;
    }
    if (!e && out_n > c->bat_out_cap) {
        e = dalloc(&c->bat_out, out_n);
        c->bat_out_cap = e ? 0 : out_n;
    }
    if (e) return from_cuda(e);
    float *di = c->bat_in, *dcf = di, *dct = di + B * n_t, *dt = di + 2 * B * n_t, *dtg = dt + B * K;
    float *dl = c->bat_out, *dcf_o = dl + B, *dct_o = dcf_o + B * n_t, *dt_o = dct_o + B * n_t,
          *dx_o = dt_o + B * K;
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
    e = cudaMemcpyAsync(dcf, cf, sizeof(float) * B * n_t, h2d, c->stream);
    if (!e) e = cudaMemcpyAsync(dct, ct, sizeof(float) * B * n_t, h2d, c->stream);
    if (!e && t) e = cudaMemcpyAsync(dt, t, sizeof(float) * B * K, h2d, c->stream);
    if (!e) e = cudaMemcpyAsync(dtg, target, sizeof(float) * B * NT, h2d, c->stream);
    if (e) return from_cuda(e);
    gbp_status st = gbp_forward_backward_batch(c, B, opts, tmpl, precision, dcf, dct, t ? dt : nullptr, dtg, dl,
                                               nullptr, dcf_o, dct_o, dt_o, dx_o);
    if (st) return st;
    if (loss) e = cudaMemcpyAsync(loss, dl, sizeof(float) * B, d2h, c->stream);
    if (!e && d_cf) e = cudaMemcpyAsync(d_cf, dcf_o, sizeof(float) * B * n_t, d2h, c->stream);
    if (!e && d_ct) e = cudaMemcpyAsync(d_ct, dct_o, sizeof(float) * B * n_t, d2h, c->stream);
    if (!e && d_t) e = cudaMemcpyAsync(d_t, dt_o, sizeof(float) * B * K, d2h, c->stream);
    if (!e && d_x) e = cudaMemcpyAsync(d_x, dx_o, sizeof(float) * B * d * K, d2h, c->stream);
    if (e) return from_cuda(e);
    return latched(c);
}

gbp_status gbp_local_solve_batch(gbp_ctx *c, int64_t n, const float *e, const float *fib, const float *cf,
                                 const float *ct, const float *Phi, int32_t mode, int32_t n_f, float *value,
                                 float *alpha)
{
    if (!c || n < 1 || !e || !fib || !cf || !ct || !Phi || !value || !alpha) return GBP_ERR_INVALID_ARG;
    if (mode != GBP_LOCAL_EXACT && mode != GBP_LOCAL_FISTA) return GBP_ERR_INVALID_ARG;
    if (mode == GBP_LOCAL_FISTA && (n_f < 1 || n_f > 256)) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaError_t err = cudaMemsetAsync(c->ctl, 0, offsetof(Control, param_status), c->stream);
    if (!err) err = gbp::launch_local_batch(c, n, e, fib, cf, ct, Phi, mode, n_f, value, alpha);
    return from_cuda(err);
}

gbp_status gbp_get_solution(gbp_ctx *c, int32_t b, float *phi, int32_t *parent, float *alpha)
{
    if (!c || (!phi && !parent && !alpha)) return GBP_ERR_INVALID_ARG;
    if (c->rec_nb < 1) return GBP_ERR_STATE;
    if (b < 0 || b >= c->rec_nb) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return from_cuda(gbp::launch_export_solution(c, b, phi, parent, alpha));
}

gbp_status gbp_diag_barrier_timeout(gbp_ctx *c, int32_t absent_ctas, int32_t max_spins)
{
    if (!c || absent_ctas < 0 || max_spins < 1) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (absent_ctas >= c->num_sms) return GBP_ERR_INVALID_ARG;
    return from_cuda(gbp::launch_barrier_probe(c, absent_ctas, (unsigned int)max_spins));
}

gbp_status gbp_enable_timing(gbp_ctx *c, int32_t on)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!on) gbp::flush_timing(c);
    c->timing = on != 0;
    return GBP_OK;
}

gbp_status gbp_get_kernel_times(gbp_ctx *c, int32_t n_classes, double *ms, int64_t *launches)
{
    if (!c || n_classes < 1 || n_classes > 8) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    gbp::flush_timing(c);
    for (int i = 0; i < n_classes; ++i) {
        if (ms) ms[i] = c->ms[i];
        if (launches) launches[i] = c->cls_launches[i];
    }
    return GBP_OK;
}

gbp_status gbp_reset_kernel_times(gbp_ctx *c)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    gbp::flush_timing(c);
    for (int i = 0; i < 8; ++i) {
        c->ms[i] = 0.0;
        c->cls_launches[i] = 0;
    }
    return GBP_OK;
}

int64_t gbp_launch_count(gbp_ctx *c) { return c ? c->launches : 0; }

gbp_status gbp_enable_trace(gbp_ctx *c, int32_t on)
{
    if (!c) return GBP_ERR_INVALID_ARG;
    c->trace_on = on != 0;
    return GBP_OK;
}

int32_t gbp_get_trace(gbp_ctx *c, int64_t *out, int32_t max_rows)
{
    if (!c || !out || max_rows < 1 || !c->trace) return 0;
    DeviceGuard g(c->device);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return 0;
    const int rows = max_rows < c->trace_cap ? max_rows : c->trace_cap;
    if (cudaMemcpy(out, c->trace, sizeof(long long) * 2 * rows, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    int n = 0;
    while (n < rows && out[2 * n + 1] != 0) ++n;
    return n;
}

}  // extern "C"
