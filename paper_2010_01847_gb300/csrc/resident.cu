// Cluster-resident stream-collide for small lattices: many time steps in
// one launch, the whole state in the shared memory of one thread-block
// cluster.
//
// A lattice of a few thousand to a few tens of thousands of nodes (the
// paper's own test lattices, 3 x 301 to 201 x 201; the 128 x 32 channel; the
// 4096 x 4 second-sound line) does too little work per step to fill the GPU:
// one launch per step costs more than the step.  Here one cluster of up to
// 16 CTAs holds both post-collision buffers (8 planes each) in shared
// memory.  CTA r owns a slab of the lattice (columns [r w, (r + 1) w) when
// nx >= ny, else rows) plus one ghost column (row) on each side.  Each step
// every CTA pulls its nodes from the current buffer (its slab and ghosts),
// applies the seam jump, walls and sides (each node's pull worked out once
// per launch with the rules of pull_node_with), collides (the collide of
// every other kernel: identical bits) and writes the other buffer; its edge
// nodes also send the populations that leave the slab into the neighbours'
// ghosts with asynchronous remote stores (st.async through distributed
// shared memory) that count their bytes on an mbarrier of the receiver.
// Before the next step a CTA waits only for its own ghost bytes (and its own
// threads, __syncthreads): no cluster-wide barrier per step.
// Global memory is read once at the start and written once at the end:
// post-collision state of the last step and of the one before it, as
// step-by-step launches would leave them (the read-outs pull from the
// latter).
//
// Every mbarrier wait is bounded (about 2 s) and reports through a status
// word (LBM_ETIMEOUT); the only cluster barriers are the one after the
// initial load and the one before exit, which every thread reaches.
#include <algorithm>

#include "lbm_kernels.h"
#include "mbarrier.cuh"

namespace plbm {
namespace {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

__device__ __forceinline__ float ld_cluster(uint32_t local_addr, unsigned rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote));
    return v;
}

// Ghost exchange between neighbouring CTAs: each edge node sends the
// populations that leave its slab with an asynchronous remote store whose
// completion counts bytes on an mbarrier of the receiving CTA; the receiver
// waits for its bytes (bounded) before it next pulls from its ghosts.
__device__ __forceinline__ uint32_t map_to(uint32_t local_addr, unsigned rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
    return remote;
}
__device__ __forceinline__ void st_async(uint32_t remote_addr, float v, uint32_t remote_bar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
            remote_addr),
        "r"(__float_as_uint(v)), "r"(remote_bar)
        : "memory");
}
// The bounded wait for a buffer's ghost bytes (about 2 s): false when it
// gave up, after setting STATUS_RESIDENT in *status (LBM_ETIMEOUT).
__device__ __forceinline__ bool ghost_wait(uint64_t *bar, uint32_t parity, int *status) {
    return mbar_wait<true>(bar, parity, status, STATUS_RESIDENT);
}

// Slab geometry shared by every CTA of the cluster.  A slab is stored with
// one ghost column (part_x) or ghost row on each side: population i of local
// node (lx, ly), lx in [-1, wx] and ly in [0, ny) for column slabs, sits at
// ((buf 8 + i) rows + ly + gy) cols + lx + gx.
struct Slabs {
    int nx, ny;
    int part_x;     // 1: slabs of columns, 0: slabs of rows
    int w;          // columns (rows) per slab; the last slabs may hold fewer or none
    int rows, cols; // allocated rows and columns of a slab plane (ghosts included)
    int nr;         // CTAs in the cluster
    int last_rank;  // the last CTA with nodes
};

template <int NPT>
__global__ void __launch_bounds__(1024, 1)
step_resident(const float *src, float *out_last, float *out_prev, long long plane, Slabs g,
              int bc_x, int bc_y, Coef<float> k, long steps, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    // after the two buffers: one mbarrier per buffer for its incoming ghosts
    uint64_t *full = reinterpret_cast<uint64_t *>(
        smem_raw + (((size_t)16 * g.rows * g.cols * sizeof(float) + 15) & ~(size_t)15));
    const int rank = (int)cluster_rank();
    const int nx = g.nx, ny = g.ny;
    const bool px = g.part_x != 0;
    const bool ghosts = g.nr > 1;
    // this CTA's slab: [x0, x0 + wx) x [y0, y0 + wy)
    const int x0 = px ? rank * g.w : 0;
    const int y0 = px ? 0 : rank * g.w;
    const int wx = px ? max(0, min(g.w, nx - x0)) : nx;
    const int wy = px ? ny : max(0, min(g.w, ny - y0));
    const int count = wx * wy;
    const int gx = px ? 1 : 0, gy = px ? 0 : 1;
    // 32-bit offsets: a CTA's shared memory holds fewer than 2^16 floats
    auto at = [&](int buf, int i, int lx, int ly) -> float * {
        return sm + (((buf * 8 + i) * g.rows + (ly + gy)) * g.cols + (lx + gx));
    };
    // this thread's nodes (fixed for the whole launch)
    int nlx[NPT], nly[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int l = threadIdx.x + j * blockDim.x;
        nly[j] = l < count ? l / wx : -1;        // -1: no node
        nlx[j] = l < count ? l - nly[j] * wx : 0;
    }

    // Fills buffer b's ghosts from the neighbouring slabs (distributed shared
    // memory): for column slabs, column x0 - 1 for the populations that
    // move right (c_x = +1) and column x0 + wx for those that move left; for
    // row slabs, the rows below and above for c_y = +1 / -1.  Periodic wrap
    // across the lattice edge; a side or wall there is never pulled from.
    auto fill_ghosts = [&](int b) {
        if (!ghosts || count == 0) return;
        const int across = px ? ny : nx;
        const int lo_owner = px ? (x0 == 0 ? g.last_rank : rank - 1)
                                : (y0 == 0 ? g.last_rank : rank - 1);
        const int lo_src = px ? (x0 == 0 ? nx - 1 : x0 - 1) : (y0 == 0 ? ny - 1 : y0 - 1);
        const int hi_edge = px ? x0 + wx : y0 + wy;
        const int hi_owner = hi_edge == (px ? nx : ny) ? 0 : rank + 1;
        const int hi_src = hi_edge == (px ? nx : ny) ? 0 : hi_edge;
        for (int t = threadIdx.x; t < 6 * across; t += blockDim.x) {
            const int side = t / (3 * across);            // 0: low ghost, 1: high ghost
            const int r = t - side * 3 * across;
            const int q = r / across, u = r - q * across;  // population slot, row / column
            // low ghost: populations moving up the partition axis (+1), high: -1
            const int i = px ? (side == 0 ? (q == 0 ? 0 : q == 1 ? 4 : 7)
                                          : (q == 0 ? 2 : q == 1 ? 5 : 6))
                             : (side == 0 ? (q == 0 ? 1 : q == 1 ? 4 : 5)
                                          : (q == 0 ? 3 : q == 1 ? 6 : 7));
            const int owner = side == 0 ? lo_owner : hi_owner;
            const int src_g = side == 0 ? lo_src : hi_src;          // global column / row
            const int src_l = src_g - owner * g.w;                  // in the owner's slab
            float *mine = px ? at(b, i, side == 0 ? -1 : wx, u) : at(b, i, u, side == 0 ? -1 : wy);
            float *theirs = px ? at(b, i, src_l, u) : at(b, i, u, src_l);
            *mine = ld_cluster((uint32_t)__cvta_generic_to_shared(theirs), (unsigned)owner);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int l = threadIdx.x; l < count; l += blockDim.x) {
        const int ly = l / wx, lx = l - ly * wx;
        const long long node = (long long)(y0 + ly) * nx + (x0 + lx);
#pragma unroll
        for (int i = 0; i < 8; ++i) *at(0, i, lx, ly) = src[(long long)i * plane + node];
    }
    // every slab loaded and every barrier initialised (and every CTA of the
    // cluster running) before any CTA reads or writes another's
    cluster_sync();
    fill_ghosts(0);
    __syncthreads();

    // the neighbouring slabs this slab sends its edge nodes to, and where
    const int lo_owner = px ? (x0 == 0 ? g.last_rank : rank - 1)
                            : (y0 == 0 ? g.last_rank : rank - 1);
    const int hi_owner = (px ? x0 + wx == nx : y0 + wy == ny) ? 0 : rank + 1;
    const int last_w = (px ? nx : ny) - g.last_rank * g.w;      // the last slab's width
    const int lo_w = (px ? x0 == 0 : y0 == 0) ? last_w : g.w;    // lo_owner's width

    // Each node's pull, worked out once for the whole launch with the rules
    // of pull_node_with (lbm_device.cuh): for population i the offset of its
    // source within a plane (own slab, ghost, or wrapped within a single
    // slab), whether it is unknown (beyond a wall or side: filled by Eq. 58 /
    // Section 2.5), and whether the node's pulls cross the seam (Eqs. 59-60).
    // info bits: 0-7 unknown i; 8 seam at x = 0 (+jump on c_x = +1); 9 seam
    // at x = nx - 1 (-jump on c_x = -1); 10 / 11 wall row bottom / top;
    // 12-15 on the left / right / bottom / top side.
    const bool walls = bc_y == BC_WALLS;
    const bool sides_x = bc_x == BC_SIDES, sides_y = bc_y == BC_SIDES;
    const bool open_y = walls || sides_y, grad = bc_x == BC_GRADIENT;
    const int pb = g.rows * g.cols;                 // one plane of a slab buffer
    unsigned rel[NPT][4], info[NPT];
    int own[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int lx = nlx[j], ly = nly[j], x = x0 + lx, y = y0 + ly;
        own[j] = (ly + gy) * g.cols + (lx + gx);
        unsigned f = 0;
        if (grad && x == 0) f |= 1u << 8;
        if (grad && x == nx - 1) f |= 1u << 9;
        if (walls && y == 0) f |= 1u << 10;
        if (walls && y == ny - 1) f |= 1u << 11;
        if (sides_x && x == 0) f |= 1u << 12;
        if (sides_x && x == nx - 1) f |= 1u << 13;
        if (sides_y && y == 0) f |= 1u << 14;
        if (sides_y && y == ny - 1) f |= 1u << 15;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int cx = cx_of(i), cy = cy_of(i);
            int sy = y - cy, sx = x - cx;
            const bool unknown = (open_y && (sy < 0 || sy >= ny)) ||
                                 (sides_x && (sx < 0 || sx >= nx));
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            int qx = sx, qy = sy;                    // source in local coordinates
            if (ghosts) {
                if (px) qx = lx - cx;
                else qy = ly - cy;
            }
            const unsigned r = unknown ? 0u : (unsigned)((qy + gy) * g.cols + (qx + gx));
            if (unknown) f |= 1u << i;
            if (i & 1) rel[j][i >> 1] |= r << 16;
            else rel[j][i >> 1] = r;
        }
        info[j] = nly[j] < 0 ? 0u : f;
    }

    // bytes of ghosts the two neighbours send into this slab per step: 3
    // populations of every node of their edge column (row) each
    const uint32_t ghost_bytes = 2u * 3u * (uint32_t)(px ? ny : nx) * (uint32_t)sizeof(float);
    const bool exchange = ghosts && count > 0;
    // the neighbours' barriers of buffers 0 and 1
    uint32_t lo_bar0 = 0u, lo_bar1 = 0u, hi_bar0 = 0u, hi_bar1 = 0u;
    if (exchange) {
        lo_bar0 = map_to(smem_u32(&full[0]), (unsigned)lo_owner);
        lo_bar1 = map_to(smem_u32(&full[1]), (unsigned)lo_owner);
        hi_bar0 = map_to(smem_u32(&full[0]), (unsigned)hi_owner);
        hi_bar1 = map_to(smem_u32(&full[1]), (unsigned)hi_owner);
    }

    bool gave_up = false, aborted = false;
    for (long s = 0; s < steps; ++s) {
        const float *A = sm + (s & 1) * 8 * pb;
        float *B = sm + ((s & 1) ^ 1) * 8 * pb;
        const int b = (int)((s & 1) ^ 1);
        // ghosts are exchanged for the steps that follow within this launch
        const bool more = s + 1 < steps;
        const uint32_t lo_bar = b ? lo_bar1 : lo_bar0, hi_bar = b ? hi_bar1 : hi_bar0;
        if (exchange && more && threadIdx.x == 0) mbar_expect_tx(&full[b], ghost_bytes);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (nly[j] < 0) continue;
            const unsigned f = info[j];
            float d[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (f & (1u << i)) {
                    d[i] = 0.f;
                } else {
                    const unsigned r = (i & 1) ? rel[j][i >> 1] >> 16 : rel[j][i >> 1] & 0xffffu;
                    float jump = 0.f;             // added as pull_node_with adds it
                    if (cx_of(i) > 0 && (f & (1u << 8))) jump = i < 4 ? k.jump_axis : k.jump_diag;
                    if (cx_of(i) < 0 && (f & (1u << 9)))
                        jump = -(i < 4 ? k.jump_axis : k.jump_diag);
                    d[i] = A[i * pb + (int)r] + jump;
                }
            }
            if (f & (1u << 10)) wall_bottom(d, k);
            if (f & (1u << 11)) wall_top(d, k);
            if (f & (0xfu << 12))
                apply_sides(d, k, (f >> 12) & 1u, (f >> 13) & 1u, (f >> 14) & 1u, (f >> 15) & 1u);
            collide(d, k);
#pragma unroll
            for (int i = 0; i < 8; ++i) B[i * pb + own[j]] = d[i];
            if (exchange && more) {
                // edge nodes also go to the neighbours' ghosts of buffer b: the
                // populations that move out of this slab towards them
                const int lx = nlx[j], ly = nly[j];
                auto send = [&](int i, int glx, int gly, int owner, uint32_t bar) {
                    st_async(map_to(smem_u32(at(b, i, glx, gly)), (unsigned)owner), d[i], bar);
                };
                if (px) {
                    if (lx == 0) { send(2, lo_w, ly, lo_owner, lo_bar);
                                   send(5, lo_w, ly, lo_owner, lo_bar);
                                   send(6, lo_w, ly, lo_owner, lo_bar); }
                    if (lx == wx - 1) { send(0, -1, ly, hi_owner, hi_bar);
                                        send(4, -1, ly, hi_owner, hi_bar);
                                        send(7, -1, ly, hi_owner, hi_bar); }
                } else {
                    if (ly == 0) { send(3, lx, lo_w, lo_owner, lo_bar);
                                   send(6, lx, lo_w, lo_owner, lo_bar);
                                   send(7, lx, lo_w, lo_owner, lo_bar); }
                    if (ly == wy - 1) { send(1, lx, -1, hi_owner, hi_bar);
                                        send(4, lx, -1, hi_owner, hi_bar);
                                        send(5, lx, -1, hi_owner, hi_bar); }
                }
            }
        }
        // this CTA's writes of step s before any of its threads reads them;
        // the same barrier tells every thread whether a wait of the step
        // before gave up, so that all of them leave the loop together
        if (__syncthreads_or(gave_up)) {
            aborted = true;
            break;
        }
        // and the neighbours' ghosts of buffer b, the (s >> 1)-th use of its
        // barrier.  A neighbour writes these ghosts again only two steps
        // later, after it has received this CTA's edge nodes of step s + 1,
        // which are sent after they were pulled from the ghosts.
        if (exchange && more) gave_up = !ghost_wait(&full[b], (uint32_t)((s >> 1) & 1), status);
    }

    // post-collision state of the last step (buffer steps & 1) and of the
    // step before it (the other buffer).  After a wait gave up the state is
    // not valid (the status word says so): nothing is written, no more
    // ghosts are sent or awaited, and the CTA goes straight to the final
    // barrier, so a stalled exchange costs one wait limit per launch.
    const int last = (int)(steps & 1);
    for (int l = threadIdx.x; l < count && !aborted; l += blockDim.x) {
        const int ly = l / wx, lx = l - ly * wx;
        const long long node = (long long)(y0 + ly) * nx + (x0 + lx);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            out_last[(long long)i * plane + node] = *at(last, i, lx, ly);
            out_prev[(long long)i * plane + node] = *at(last ^ 1, i, lx, ly);
        }
    }
    // no CTA may leave while another can still read its shared memory (the
    // last step sends no ghosts, so no remote store is in flight)
    cluster_sync();
}

constexpr int MAX_CLUSTER = 16;
constexpr int THREADS = 1024;
constexpr int MAX_NPT = 4;            // nodes per thread
constexpr int NODES_PER_CTA = 256;    // spread the lattice over up to 16 SMs

struct DevState {
    bool ready = false;
    int optin = 0, cap = 0;
};
DevState g_dev[64];

template <int NPT> constexpr auto kernel_npt() { return step_resident<NPT>; }
using KernelFn = void (*)(const float *, float *, float *, long long, Slabs, int, int,
                          Coef<float>, long, int *);
KernelFn kernel_of(int npt) {
    switch (npt) {
        case 1: return kernel_npt<1>();
        case 2: return kernel_npt<2>();
        case 3: return kernel_npt<3>();
        default: return kernel_npt<4>();
    }
}

// Once per device: clusters of up to 16 CTAs, and the largest dynamic
// shared memory a plan may ask for (plans of several lattices coexist).
cudaError_t prepare(int dev) {
    DevState &d = g_dev[dev];
    if (d.ready) return cudaSuccess;
    cudaError_t e = cudaDeviceGetAttribute(&d.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    d.cap = d.optin - 1024;                           // bytes per CTA (some kept spare)
    for (int npt = 1; npt <= MAX_NPT; ++npt) {
        e = cudaFuncSetAttribute(kernel_of(npt), cudaFuncAttributeNonPortableClusterSizeAllowed,
                                 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kernel_of(npt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 d.cap);
        if (e != cudaSuccess) return e;
    }
    d.ready = true;
    return cudaSuccess;
}

cudaLaunchConfig_t config_of(const ResidentPlan &p, cudaLaunchAttribute *attr,
                             cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)p.threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)p.smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

cudaError_t resident_plan(int precision, int nx, int ny, int cluster_req, ResidentPlan *out) {
    *out = ResidentPlan{};
    if (precision != PREC_FP32 || nx < 1 || ny < 1) return cudaErrorNotSupported;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if ((e = prepare(dev)) != cudaSuccess) return e;
    const int cap = g_dev[dev].cap;
    const long long plane = (long long)nx * ny;
    const int part_x = nx >= ny ? 1 : 0;
    const int extent = part_x ? nx : ny, across = part_x ? ny : nx;
    const int most = std::min(MAX_CLUSTER, extent);   // at least one column (row) per CTA
    // about NODES_PER_CTA nodes per CTA (the work of a step spread over up to
    // 16 SMs), then larger clusters (less shared memory each), then smaller
    int want = (int)std::min<long long>(most, (plane + NODES_PER_CTA - 1) / NODES_PER_CTA);
    if (cluster_req > 0) want = std::min(cluster_req, most);
    if (want < 1) want = 1;
    int order[MAX_CLUSTER];
    int n_order = 0;
    for (int nr = want; nr <= most; ++nr) order[n_order++] = nr;
    for (int nr = want - 1; nr >= 1; --nr) order[n_order++] = nr;
    if (cluster_req > 0) n_order = 1;
    for (int oi = 0; oi < n_order; ++oi) {
        const int nr = order[oi];
        const int w = (extent + nr - 1) / nr;
        const long long nodes = (long long)w * across;              // per CTA, at most
        const int threads = (int)std::min<long long>(THREADS, (nodes + 31) / 32 * 32);
        const long long npt = (nodes + threads - 1) / threads;
        if (npt > MAX_NPT) continue;
        const int rows = part_x ? ny : w + 2, cols = part_x ? w + 2 : nx;
        // two buffers, then two mbarriers (16-byte aligned)
        const long long bytes =
            ((2LL * 8 * rows * cols * (long long)sizeof(float) + 15) & ~15LL) + 16;
        if (bytes > cap) continue;
        ResidentPlan p;
        p.cluster = nr;
        p.part_x = part_x;
        p.w = w;
        p.rows = rows;
        p.cols = cols;
        p.last_rank = (extent - 1) / w;
        p.npt = (int)npt;
        p.threads = threads;
        p.smem = (int)bytes;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = config_of(p, attr, nullptr);
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, kernel_of(p.npt), &cfg);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (clusters < 1) continue;
        *out = p;
        return cudaSuccess;
    }
    return cudaErrorNotSupported;
}

namespace {

// The resident kernel's ghost wait on a fresh barrier that nothing
// completes, in one thread of a one-CTA cluster: the wait gives up at its
// limit (about 2 s) and sets STATUS_RESIDENT in *status, exactly as a
// stalled ghost exchange would.
__global__ void __cluster_dims__(1, 1, 1) resident_wait_probe(int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) ghost_wait(&bar, 0u, status);
}

}  // namespace

cudaError_t launch_resident_wait_probe(int *status, cudaStream_t stream) {
    resident_wait_probe<<<1, 32, 0, stream>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_resident(const float *src, float *out_last, float *out_prev, int nx, int ny,
                            int bc_x, int bc_y, const Coef<float> &k, long steps,
                            const ResidentPlan &p, int *status, cudaStream_t stream) {
    if (p.cluster < 1 || p.npt < 1 || p.npt > MAX_NPT) return cudaErrorInvalidConfiguration;
    if (steps < 1) return cudaSuccess;
    Slabs g{nx, ny, p.part_x, p.w, p.rows, p.cols, p.cluster, p.last_rank};
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config_of(p, attr, stream);
    return cudaLaunchKernelEx(&cfg, kernel_of(p.npt), src, out_last, out_prev,
                              (long long)nx * ny, g, bc_x, bc_y, k, steps, status);
}

}  // namespace plbm
