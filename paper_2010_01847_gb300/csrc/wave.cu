// Multi-step stream-collide kernel: K time steps of Eq. 13 per pass over
// the population planes in HBM (temporal blocking, FP32 storage).  One warp
// per strip-segment of the lattice; the march is in wave.cuh.
#include "lbm_kernels.h"
#include "wave.cuh"

namespace plbm {
namespace {

using wave::Strip;

// one strip per block: 32-thread blocks (12 per SM at 156 registers) ran the
// 4-step kernel at 354.5 GLUPS at 8192^2, against 324.4 with 2 warps per block
// and 320.3 with 4 (the same warps per SM)
constexpr int WAVE_WARPS = 1;
constexpr int WAVE_SMEM = WAVE_WARPS * wave::RING_ELEMS * (int)sizeof(float2);

template <int K, bool SEAM, bool WALLS>
__global__ void __launch_bounds__(WAVE_WARPS * 32)
step_wave(const Strip a, const Coef<float> k, int tiles_x, long long items) {
    extern __shared__ float2 wave_ring[];
    const long long item = (long long)blockIdx.x * WAVE_WARPS + (threadIdx.x >> 5);
    if (item >= items) return;                   // whole warps leave together
    wave::run_strip<K, SEAM, WALLS>(a, k, int(item % tiles_x), int(item / tiles_x), wave::halo(K),
                             wave_ring + (threadIdx.x >> 5) * wave::RING_ELEMS);
}

template <int K>
cudaError_t launch_k(const Strip &a, const Coef<float> &k, cudaStream_t stream) {
    const int S = wave::stride_of(wave::halo(K));
    const int tiles_x = (a.nx + S - 1) / S;
    const long long segs = (a.ny + a.seg_rows - 1) / a.seg_rows;
    const long long items = (long long)tiles_x * segs;
    const long long blocks = (items + WAVE_WARPS - 1) / WAVE_WARPS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned g = (unsigned)blocks;
    const bool seam = a.bc_x == BC_GRADIENT, walls = a.bc_y == BC_WALLS;
    if (seam && walls)
        step_wave<K, true, true><<<g, WAVE_WARPS * 32, WAVE_SMEM, stream>>>(a, k, tiles_x, items);
    else if (seam)
        step_wave<K, true, false><<<g, WAVE_WARPS * 32, WAVE_SMEM, stream>>>(a, k, tiles_x, items);
    else if (walls)
        step_wave<K, false, true><<<g, WAVE_WARPS * 32, WAVE_SMEM, stream>>>(a, k, tiles_x, items);
    else
        step_wave<K, false, false><<<g, WAVE_WARPS * 32, WAVE_SMEM, stream>>>(a, k, tiles_x, items);
    return cudaGetLastError();
}

}  // namespace

bool wave_supported(int precision, int nx, int ny, int bc_x, int bc_y) {
    (void)ny;
    const bool bc_ok = (bc_x == BC_PERIODIC || bc_x == BC_GRADIENT) &&
                       (bc_y == BC_PERIODIC || bc_y == BC_WALLS);
    if (precision == PREC_FP32) return bc_ok && nx >= 2 && nx % 2 == 0;
    // 16-bit storage: tiles of 8 nodes (4 lanes of a strip)
    if (has_tile_refs(precision)) return bc_ok && nx >= 8 && nx % 8 == 0;
    return false;
}

int wave_max_steps(int precision) {
    return precision == PREC_FP32 ? WAVE_MAX_STEPS : WAVE16_MAX_STEPS;
}

cudaError_t launch_step_wave(int steps, const float *src, float *dst, int nx, int ny, int bc_x,
                             int bc_y, const Coef<float> &k, int seg_rows, cudaStream_t stream) {
    if (!wave_supported(PREC_FP32, nx, ny, bc_x, bc_y) || steps < WAVE_MIN_STEPS ||
        steps > WAVE_MAX_STEPS || seg_rows < 1 || src == dst)
        return cudaErrorInvalidValue;
    Strip a;
    a.src = src;
    a.dst = dst;
    a.plane = (long long)nx * ny;
    a.nx = nx;
    a.ny = ny;
    a.bc_x = bc_x;
    a.bc_y = bc_y;
    a.seg_rows = seg_rows < ny ? seg_rows : ny;
    switch (steps) {
        case 2: return launch_k<2>(a, k, stream);
        case 3: return launch_k<3>(a, k, stream);
        case 4: return launch_k<4>(a, k, stream);
        case 5: return launch_k<5>(a, k, stream);
        case 6: return launch_k<6>(a, k, stream);
        case 7: return launch_k<7>(a, k, stream);
        default: return launch_k<8>(a, k, stream);
    }
}

}  // namespace plbm
