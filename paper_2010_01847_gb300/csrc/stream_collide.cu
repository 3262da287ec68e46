// Fused pull-stream + boundary + collision kernels: one launch is one time
// step of Eq. 13 over the whole lattice.
//
// The kernels read the post-collision planes of step n-1 (`src`), pull the
// populations arriving at each node (left-hand side of Eq. 13, seam jump of
// Eqs. 59-60, diffuse walls of Eq. 58), collide them in registers
// (Eqs. 15, 16, 53, 54) and write the post-collision planes of step n
// (`dst`).  Layout: structure of arrays, 8 planes of ny*nx, x fastest.
// With RES the kernel also accumulates the residual sums of the pulled state
// (the state at step n) and writes one set of 5 partial sums per block.
#include "lbm_kernels.h"

namespace plbm {

// ---------------------------------------------------------------------------
// Scalar kernel: one thread per node, any nx.  Serves ragged lattices (nx not
// a multiple of the vector width) and is the simplest statement of the step.
template <typename T, bool RES>
__global__ void __launch_bounds__(256)
step_scalar(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
            long long plane, int bc_x, int bc_y, Coef<typename Store<T>::C> k,
            ResidualReq<typename Store<T>::C> rq) {
    using C = typename Store<T>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (node < plane) {
        const int y = int(node / nx);
        const int x = int(node - (long long)y * nx);
        C d[8];
        pull_node<T>(src, plane, nx, ny, x, y, bc_x, bc_y, k, d);
        if (RES) residual_node(d, k, rq.inv_scale, rq.prev, plane, node, rq.have_prev != 0, acc);
        collide(d, k);
#pragma unroll
        for (int i = 0; i < 8; ++i) dst[(long long)i * plane + node] = Store<T>::put(d[i]);
    }
    if (RES) block_sum5_store(acc, rq.partials + (size_t)blockIdx.x * 5);
}

// ---------------------------------------------------------------------------
// 16-byte vector packing of V = 16/sizeof(T) consecutive plane elements.
template <typename T> struct Pack;
template <> struct Pack<float> {
    static constexpr int V = 4;
    __device__ static void unpack(uint4 r, float (&o)[4]) {
        o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
    }
    __device__ static uint4 pack(const float (&o)[4]) {
        return make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]),
                          __float_as_uint(o[2]), __float_as_uint(o[3]));
    }
};
template <> struct Pack<double> {
    static constexpr int V = 2;
    __device__ static void unpack(uint4 r, double (&o)[2]) {
        o[0] = __hiloint2double((int)r.y, (int)r.x);
        o[1] = __hiloint2double((int)r.w, (int)r.z);
    }
    __device__ static uint4 pack(const double (&o)[2]) {
        return make_uint4((unsigned)__double2loint(o[0]), (unsigned)__double2hiint(o[0]),
                          (unsigned)__double2loint(o[1]), (unsigned)__double2hiint(o[1]));
    }
};
template <> struct Pack<__half> {
    static constexpr int V = 8;
    __device__ static float2 w2f(unsigned w) {
        __half2 h = *reinterpret_cast<__half2 *>(&w);
        return __half22float2(h);
    }
    __device__ static unsigned f2w(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<unsigned *>(&h);
    }
    __device__ static void unpack(uint4 r, float (&o)[8]) {
        float2 a = w2f(r.x), b = w2f(r.y), c = w2f(r.z), d = w2f(r.w);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
    }
    __device__ static uint4 pack(const float (&o)[8]) {
        return make_uint4(f2w(o[0], o[1]), f2w(o[2], o[3]), f2w(o[4], o[5]), f2w(o[6], o[7]));
    }
};
template <> struct Pack<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ static float2 w2f(unsigned w) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
        return __bfloat1622float2(h);
    }
    __device__ static unsigned f2w(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<unsigned *>(&h);
    }
    __device__ static void unpack(uint4 r, float (&o)[8]) {
        float2 a = w2f(r.x), b = w2f(r.y), c = w2f(r.z), d = w2f(r.w);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
    }
    __device__ static uint4 pack(const float (&o)[8]) {
        return make_uint4(f2w(o[0], o[1]), f2w(o[2], o[3]), f2w(o[4], o[5]), f2w(o[6], o[7]));
    }
};

__device__ __forceinline__ uint4 ld_stream(const void *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ void st_stream(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Vector kernel: each thread owns V consecutive nodes of one row and moves
// every plane with one aligned 16-byte load and one 16-byte store.  The
// x-shifted populations (c_x = +-1) take their out-of-vector neighbour from
// the adjacent lane by a warp shuffle; the first/last lane of a warp, and
// rows' ends, load that one element directly (wrapping at the seam).
// Requires nx % V == 0.  Threads are laid out row-major over the lattice,
// so a warp may straddle two rows; the row test handles that.
template <typename T, bool RES>
__global__ void __launch_bounds__(256)
step_vector(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
            long long plane, int bc_x, int bc_y, Coef<typename Store<T>::C> k,
            ResidualReq<typename Store<T>::C> rq) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const int tpr = nx / V;
    const long long total = (long long)tpr * ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < total;
    const int y = active ? int(t / tpr) : 0;
    const int xv = active ? int(t - (long long)y * tpr) : 0;
    const int x0 = xv * V;
    const int lane = threadIdx.x & 31;
    const bool walls = bc_y == BC_WALLS;
    const bool bottom = walls && y == 0;
    const bool top = walls && y == ny - 1;

    C d[8][V];
    long long row_off[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cy = cy_of(i);
        int sy = y - cy;
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        row_off[i] = (long long)i * plane + (long long)sy * nx;
        const bool unknown = (cy > 0 && bottom) || (cy < 0 && top);
        if (active && !unknown) {
            Pack<T>::unpack(ld_stream(src + row_off[i] + x0), d[i]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) d[i][j] = C(0);
        }
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        if (cx == 0) continue;
        const bool unknown = (cy > 0 && bottom) || (cy < 0 && top);
        const C jw = (i < 4) ? k.jump_axis : k.jump_diag;
        if (cx > 0) {
            C left = __shfl_up_sync(0xffffffffu, d[i][V - 1], 1);
            if ((lane == 0 || xv == 0) && active && !unknown) {
                int sx = x0 - 1;
                C jump = C(0);
                if (sx < 0) {
                    sx += nx;
                    if (bc_x == BC_GRADIENT) jump = jw;
                }
                left = Store<T>::load(src[row_off[i] + sx]) + jump;
            }
#pragma unroll
            for (int j = V - 1; j >= 1; --j) d[i][j] = d[i][j - 1];
            d[i][0] = left;
        } else {
            C right = __shfl_down_sync(0xffffffffu, d[i][0], 1);
            if ((lane == 31 || xv + 1 == tpr) && active && !unknown) {
                int sx = x0 + V;
                C jump = C(0);
                if (sx >= nx) {
                    sx -= nx;
                    if (bc_x == BC_GRADIENT) jump = -jw;
                }
                right = Store<T>::load(src[row_off[i] + sx]) + jump;
            }
#pragma unroll
            for (int j = 0; j < V - 1; ++j) d[i][j] = d[i][j + 1];
            d[i][V - 1] = right;
        }
    }

    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (active) {
        const long long out = (long long)y * nx + x0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            C n[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) n[i] = d[i][j];
            if (bottom) wall_bottom(n, k);
            if (top) wall_top(n, k);
            if (RES) residual_node(n, k, rq.inv_scale, rq.prev, plane, out + j,
                                   rq.have_prev != 0, acc);
            collide(n, k);
#pragma unroll
            for (int i = 0; i < 8; ++i) d[i][j] = n[i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            st_stream(dst + (long long)i * plane + out, Pack<T>::pack(d[i]));
    }
    if (RES) block_sum5_store(acc, rq.partials + (size_t)blockIdx.x * 5);
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_step(int kernel, const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                        const Coef<typename Store<T>::C> &k, int *status,
                        const ResidualReq<typename Store<T>::C> *rq, const StagedPlan &plan,
                        int *blocks_out, cudaStream_t stream) {
    const long long plane = (long long)nx * ny;
    if (kernel == KERNEL_STAGED)
        return launch_step_staged<T>(src, dst, nx, ny, bc_x, bc_y, k, status, rq, plan,
                                     blocks_out, stream);
    const ResidualReq<typename Store<T>::C> none{};
    const long long threads = kernel == KERNEL_VECTOR ? plane / Pack<T>::V : plane;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks_out) *blocks_out = (int)blocks;
    if (kernel == KERNEL_VECTOR) {
        if (rq)
            step_vector<T, true><<<blocks, 256, 0, stream>>>(src, dst, nx, ny, plane, bc_x, bc_y,
                                                             k, *rq);
        else
            step_vector<T, false><<<blocks, 256, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                              bc_y, k, none);
    } else {
        if (rq)
            step_scalar<T, true><<<blocks, 256, 0, stream>>>(src, dst, nx, ny, plane, bc_x, bc_y,
                                                             k, *rq);
        else
            step_scalar<T, false><<<blocks, 256, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                              bc_y, k, none);
    }
    return cudaGetLastError();
}

long long step_blocks(int kernel, int precision, int nx, int ny, const StagedPlan &plan) {
    const long long plane = (long long)nx * ny;
    if (kernel == KERNEL_STAGED) return plan.grid;
    const long long threads = kernel == KERNEL_VECTOR ? plane / vector_width(precision) : plane;
    return (threads + 255) / 256;
}

int vector_width(int precision) {
    switch (precision) {
        case PREC_FP32: return Pack<float>::V;
        case PREC_FP64: return Pack<double>::V;
        default: return Pack<__half>::V;
    }
}

#define PLBM_STEP(T)                                                                         \
    template cudaError_t launch_step<T>(int, const T *, T *, int, int, int, int,             \
                                        const Coef<Store<T>::C> &, int *,                    \
                                        const ResidualReq<Store<T>::C> *, const StagedPlan &, \
                                        int *, cudaStream_t);
PLBM_STEP(float)
PLBM_STEP(double)
PLBM_STEP(__half)
PLBM_STEP(__nv_bfloat16)

}  // namespace plbm
