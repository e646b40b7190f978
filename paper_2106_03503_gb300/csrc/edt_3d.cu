// 3-D exact EDT.  The paper processes the dimensions one after the other
// (Sec. 3.1: methods "based on the separate processing of all dimensions");
// for a [Dz][H][W] volume this library runs
//   (z) the column pass along z: the volume seen as a 2-D image with Dz rows
//       and H*W columns, handled by the same column-bit kernel as 2-D images;
//   (y) the lower envelope of Sec. 3.3.1 along y, over f(y') = (z - z')^2 with
//       z' the nearest source along z in column (y', x): for each voxel it
//       records the source (z', y') of its owning parabola, packed as
//       z' << 16 | y' (0xFFFFFFFF = no source in the whole x-slice);
//   (x) the lower envelope along x over f(x') = (z - z')^2 + (y - y')^2 read
//       from that record, writing D, F = z'*H*W + y'*W + x' and sqrt(D).
// The (z', y') record lives in the caller's F (or D) buffer: the x pass reads
// a row into shared memory before it overwrites the same row.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr uint32_t PNONE = 0xFFFFFFFFu;

// --- y pass ----------------------------------------------------------------

struct LineY {
    int n;                   // H
    const int* gz;           // padded [H]: nearest source z of (y', x), -1 none
    int lg;
    int z;
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        const int g = gz[pad_index(k, lg)];
        if (g < 0) return false;
        f = (z - g) * (z - g);
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        const int g = gz[pad_index(k, lg)];
        return (z - g) * (z - g) + k * k;
    }
    __device__ __forceinline__ int feature(int k) const
    {
        return (int)(((uint32_t)gz[pad_index(k, lg)] << 16) | (uint32_t)k);
    }
};

struct OutY {
    uint32_t* tile;          // [H][XT + 1]
    int TP;                  // tile pitch, XT + 1
    int xl;
    __device__ __forceinline__ void store(int j, int v, int f) const
    {
        tile[j * TP + xl] = (v == INT32_MAX) ? PNONE : (uint32_t)f;
    }
};

// One block: one z, XT consecutive x (one warp per x line).
__global__ void __launch_bounds__(1024)
k_ypass3d(int Dz, int H, int W, ColScratch s, int XT, uint32_t* __restrict__ P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lg = seg_log2(H);
    const int SW = ((1 << lg) + 31) / 32;
    const int pitch = padded_len(H) | 1;       // odd: conflict-free fills
    int* gz = reinterpret_cast<int*>(smem);    // [XT][pitch]
    const int TP = XT + 1;
    uint32_t* tile = reinterpret_cast<uint32_t*>(gz + XT * pitch);   // [H][TP]
    unsigned char* wbase = reinterpret_cast<unsigned char*>(tile + (size_t)H * TP);
    wbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(wbase) + 15) & ~uintptr_t(15));
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    const int xtiles = (W + XT - 1) / XT;
    const int z = blockIdx.x / xtiles;
    const int x0 = (blockIdx.x % xtiles) * XT;
    const int64_t plane = (int64_t)H * W;
    const int zb = z >> 5, zr = z & 31, zG = zb >> 5;

    // nearest source along z for every (y, x) of the tile
    for (int e = threadIdx.x; e < H * XT; e += blockDim.x) {
        const int y = e / XT, xl = e % XT, x = x0 + xl;
        int g = -1;
        if (x < W) {
            const int64_t p = (int64_t)y * W + x;
            const uint32_t w = s.C[(int64_t)zb * plane + p];
            const uint32_t u = s.U[(int64_t)zb * plane + p];
            uint32_t up = u & 0xFFFFu, dn = u >> 16;
            if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                const uint32_t gab = s.GAB[(int64_t)zG * plane + p];
                if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                if (dn == (uint32_t)NONE16) dn = gab >> 16;
            }
            g = nearest_in_column(w, zb * 32, zr, (int)up, (int)dn);
        }
        gz[xl * pitch + pad_index(y, lg)] = g;
    }
    __syncthreads();

    if (warp < XT && x0 + warp < W) {
        const WarpSmem sm = carve_warp_smem(wbase + warp * warp_smem_bytes(SW), SW);
        const LineY line{H, gz + warp * pitch, lg, z};
        const OutY out{tile, TP, warp};
        warp_envelope(line, out, sm);
    }
    __syncthreads();

    // coalesced write of the (z', y') records
    for (int e = threadIdx.x; e < H * XT; e += blockDim.x) {
        const int y = e / XT, xl = e % XT, x = x0 + xl;
        if (x < W) P[(int64_t)z * plane + (int64_t)y * W + x] = tile[y * TP + xl];
    }
    (void)lane;
    (void)Dz;
}

// --- x pass ----------------------------------------------------------------

struct LineX {
    int n;                   // W
    const uint32_t* rec;     // padded [W]: (z', y') records of this row
    int lg;
    int z, y, H, W;
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        const uint32_t p = rec[pad_index(k, lg)];
        if (p == PNONE) return false;
        const int dz = z - (int)(p >> 16), dy = y - (int)(p & 0xFFFFu);
        f = dz * dz + dy * dy;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        int f;
        eval(k, f);
        return f + k * k;
    }
    __device__ __forceinline__ int feature(int k) const
    {
        const uint32_t p = rec[pad_index(k, lg)];
        return ((int)(p >> 16) * H + (int)(p & 0xFFFFu)) * W + k;
    }
};

struct OutX {
    int32_t* D;
    int32_t* F;
    float* dist;
    int64_t rowoff;
    __device__ __forceinline__ void store(int j, int v, int f) const
    {
        const int64_t i = rowoff + j;
        if (D) D[i] = v;
        if (F) F[i] = f;
        if (dist) dist[i] = sqrt_rn_int(v);
    }
};

// One block: `rows` consecutive rows (z, y) ... of the volume, one warp each.
__global__ void __launch_bounds__(256)
k_xpass3d(int Dz, int H, int W, int rows, const uint32_t* P, int32_t* D,
          int32_t* F, float* dist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lg = seg_log2(W);
    const int SW = ((1 << lg) + 31) / 32;
    const int np = padded_len(W);
    uint32_t* rec = reinterpret_cast<uint32_t*>(smem);   // [rows][np]
    unsigned char* wbase = smem + (((size_t)rows * np * 4 + 15) & ~size_t(15));
    const int warp = threadIdx.x >> 5;
    const int64_t nrows = (int64_t)Dz * H;
    const int64_t row0 = (int64_t)blockIdx.x * rows;

    for (int e = threadIdx.x; e < rows * W; e += blockDim.x) {
        const int rl = e / W, k = e % W;
        const int64_t row = row0 + rl;
        if (row < nrows) rec[rl * np + pad_index(k, lg)] = P[row * W + k];
    }
    __syncthreads();

    const int64_t row = row0 + warp;
    if (warp < rows && row < nrows) {
        const WarpSmem sm = carve_warp_smem(wbase + warp * warp_smem_bytes(SW), SW);
        const int z = (int)(row / H), y = (int)(row % H);
        const LineX line{W, rec + warp * np, lg, z, y, H, W};
        const OutX out{D, F, dist, row * W};
        warp_envelope(line, out, sm);
    }
}

cudaError_t launch_ypass3d(int Dz, int H, int W, const ColGeom& g,
                           const ColScratch& s, uint32_t* P, cudaStream_t stream)
{
    (void)g;
    const int lg = seg_log2(H);
    const int SW = ((1 << lg) + 31) / 32;
    const int pitch = padded_len(H) | 1;
    int XT = 32;
    auto smem_for = [&](int xt) {
        return (size_t)xt * pitch * 4 + (size_t)H * (xt + 1) * 4 + 16 + (size_t)xt * warp_smem_bytes(SW);
    };
    while (XT > 1 && smem_for(XT) > 200 * 1024) XT >>= 1;
    const size_t smem = smem_for(XT);
    const int xtiles = (W + XT - 1) / XT;
    const unsigned blocks = (unsigned)((int64_t)Dz * xtiles);
    k_ypass3d<<<blocks, XT * 32, smem, stream>>>(Dz, H, W, s, XT, P);
    return cudaGetLastError();
}

cudaError_t launch_xpass3d(int Dz, int H, int W, uint32_t* P, int32_t* D,
                           int32_t* F, float* dist, cudaStream_t stream)
{
    const int lg = seg_log2(W);
    const int SW = ((1 << lg) + 31) / 32;
    const int np = padded_len(W);
    int rows = 8;
    while (rows > 1 && (size_t)rows * (np * 4 + warp_smem_bytes(SW)) > 200 * 1024) rows >>= 1;
    const size_t smem = (((size_t)rows * np * 4 + 15) & ~size_t(15)) + (size_t)rows * warp_smem_bytes(SW);
    const int64_t nrows = (int64_t)Dz * H;
    const unsigned blocks = (unsigned)((nrows + rows - 1) / rows);
    k_xpass3d<<<blocks, rows * 32, smem, stream>>>(Dz, H, W, rows, P, D, F, dist);
    return cudaGetLastError();
}

cudaError_t set_3d_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_ypass3d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_xpass3d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace edt
