// FP32-bulk step of a single lattice model with the neighbours' records staged
// in shared memory by TMA, one box of the lattice per thread block.
//
// The stencil step of pd_step_f32_lat.cu (the same walk, flags, near-s_c rule
// and node update, hence the same bits) for single bond-based lattice models.
// A block owns a box of BZ x BY x BX lattice nodes (z fastest, one node per
// thread).  Before its walk one thread issues a single tiled bulk tensor copy
// (cp.async.bulk.tensor, 4-D: the 4 floats of a record, z, y, x) of the
// published records of the box grown by the stencil's reach (3 nodes on every
// side) into shared memory, completed on an mbarrier; records outside the
// lattice arrive as zeros (the copy's out-of-bounds fill), the values the record
// array's zero halo holds.  The walk then reads every neighbour from shared
// memory at offsets fixed when the kernel is compiled (TZ (o_y + TY o_x) + o_z
// records from the node's own): no 64-bit neighbour address arithmetic and no
// L1 misses on the records.  Flags, the FP64 state, the near-s_c decisions and
// the node update read global memory as in the one-warp-per-32-nodes kernel.
//
// The wait on the copy is bounded (about half a second): past it the block
// sets PD_DEVERR_TIMEOUT, waits once more (bounded) so that no copy is in
// flight into its shared memory, and leaves.
#define PD_LAT_HELPERS 1
#include "pd_step_f32_lat.cu"

namespace pd {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make the barrier's initialisation visible to the copy engine (async proxy)
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier, at most kTmaWaitNs (and at most
// kTmaWaitIters polls); false if it did not complete.
constexpr uint64_t kTmaWaitNs = 500000000ull;
constexpr int kTmaWaitIters = 1 << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < kTmaWaitIters; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kTmaWaitNs) break;
    }
    return false;
}

// One tiled 4-D bulk tensor copy global -> shared, completed on `bar`
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_addr(bar))
        : "memory");
}

template <int SCM, bool PBC, int BZ, int BY, int BX>
__global__ void __launch_bounds__(BZ * BY * BX, PD_LAT_MIN_BLOCKS)
    k_step_f32_lat_tma(const __grid_constant__ StepArgsF32 a, const __grid_constant__ LatTmaArgs t)
{
    constexpr int TZ = BZ + 6, TY = BY + 6, TX = BX + 6;
    constexpr uint32_t kBytes = 16u * TZ * TY * TX;
    static_assert(kBytes == lat_tma_tile_bytes(BZ, BY, BX), "tile size");
    extern __shared__ unsigned char smem_raw[];
    // the tile at a 128-byte boundary, the barrier after it (the launch asks for
    // lat_tma_smem_bytes: the tile, 128 bytes of slack and the barrier)
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float4* tile = reinterpret_cast<float4*>(base);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + kBytes);

    const int64_t step = lat_step_of(a);
    lat_advance_counter(a);
    const int cur = (int)(step & 1);
    const int b = blockIdx.x;
    const int bz = b % t.tiles_z, by = (b / t.tiles_z) % t.tiles_y, bx = b / (t.tiles_z * t.tiles_y);
    const int z0 = bz * BZ, y0 = by * BY, x0 = bx * BX;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, kBytes + (uint32_t)t.extra_tx);
        tma_load_4d(tile, &t.map[cur], 0, z0 - 3, y0 - 3, x0 - 3, bar);
    }
    if (!mbar_wait_bounded(bar, 0)) {
        if (threadIdx.x == 0) atomicOr(a.err, PD_DEVERR_TIMEOUT);
        mbar_wait_bounded(bar, 0);
        return;
    }

    const int tz = (int)threadIdx.x % BZ, ty = ((int)threadIdx.x / BZ) % BY;
    const int tx = (int)threadIdx.x / (BZ * BY);
    const int iz = z0 + tz, iy = y0 + ty, ix = x0 + tx;
    if (iz >= t.nz || iy >= t.ny || ix >= t.nx) return;
    LatNode s;
    s.i = ((int64_t)ix * t.ny + iy) * t.nz + iz;
    s.slot0 = (s.i >> 5) * (int64_t)(kStencilSlots * 32) + (s.i & 31);
    const float4* Ti = tile + ((tz + 3) + TZ * ((ty + 3) + TY * (tx + 3)));
    lat_node_begin(s, *Ti);
    uint32_t* bw = a.bits + (s.i >> 5) * (int64_t)kStencilSlots + (s.i & 31);
    uint32_t w0[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w0[q] = s.word[q] = bw[q * 32];
    lat_walk<SrcTile<TZ, TY>, SCM, PBC>(a, cur, Ti, s);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (s.word[q] != w0[q]) bw[q * 32] = s.word[q];
    lat_update(a, s, step, a.lat_u[cur], a.lat_u[cur ^ 1], const_cast<float4*>(a.lat_pub[cur ^ 1]));
}

template <int BZ, int BY, int BX>
const void* tma_kernel(int sc_mode, bool pbc)
{
    if (pbc)
        return sc_mode == 0 ? (const void*)k_step_f32_lat_tma<0, true, BZ, BY, BX>
                            : (const void*)k_step_f32_lat_tma<1, true, BZ, BY, BX>;
    return sc_mode == 0 ? (const void*)k_step_f32_lat_tma<0, false, BZ, BY, BX>
                        : (const void*)k_step_f32_lat_tma<1, false, BZ, BY, BX>;
}

template <int BZ, int BY, int BX>
void tma_launch(const StepArgsF32& a, const LatTmaArgs& t, int sc_mode, bool pbc, int grid,
                size_t smem, cudaStream_t s)
{
    constexpr int threads = BZ * BY * BX;
    if (sc_mode == 0) {
        if (pbc) k_step_f32_lat_tma<0, true, BZ, BY, BX><<<grid, threads, smem, s>>>(a, t);
        else k_step_f32_lat_tma<0, false, BZ, BY, BX><<<grid, threads, smem, s>>>(a, t);
    } else {
        if (pbc) k_step_f32_lat_tma<1, true, BZ, BY, BX><<<grid, threads, smem, s>>>(a, t);
        else k_step_f32_lat_tma<1, false, BZ, BY, BX><<<grid, threads, smem, s>>>(a, t);
    }
}

}  // namespace

const void* step_f32_kernel_lat_tma(int shape, int sc_mode, bool per_bond_c)
{
    switch (shape) {
    case 0: return tma_kernel<16, 2, 8>(sc_mode, per_bond_c);
    case 1: return tma_kernel<8, 4, 8>(sc_mode, per_bond_c);
    default: return tma_kernel<32, 2, 4>(sc_mode, per_bond_c);
    }
}

cudaError_t launch_step_f32_lat_tma(const StepArgsF32& a, const LatTmaArgs& t, int shape,
                                    int sc_mode, int grid, cudaStream_t s)
{
    const bool pbc = a.cbond != nullptr;
    const size_t smem = lat_tma_smem_bytes(shape);
    switch (shape) {
    case 0: tma_launch<16, 2, 8>(a, t, sc_mode, pbc, grid, smem, s); break;
    case 1: tma_launch<8, 4, 8>(a, t, sc_mode, pbc, grid, smem, s); break;
    default: tma_launch<32, 2, 4>(a, t, sc_mode, pbc, grid, smem, s); break;
    }
    return cudaGetLastError();
}

}  // namespace pd
