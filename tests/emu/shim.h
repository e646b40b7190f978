// Host stand-ins for the CUDA keywords, types and intrinsics that libedt's
// kernels use, so that the kernel sources compile as C++ for the emulation
// in tests/emu (test infrastructure; never part of the library).
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <cassert>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <thread>
#include <type_traits>
#include <vector>

#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __launch_bounds__(...)
#define __grid_constant__
#define __shared__ static
#define __align__(n) alignas(n)

template <class A, class B> inline typename std::common_type<A, B>::type min(A a, B b) { return a < b ? a : b; }
template <class A, class B> inline typename std::common_type<A, B>::type max(A a, B b) { return a > b ? a : b; }

struct EmuDim { unsigned x = 0, y = 0, z = 0; };
struct dim3 { unsigned x = 1, y = 1, z = 1; dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {} };
extern thread_local EmuDim threadIdx, blockIdx, blockDim, gridDim;

struct int4 { int x, y, z, w; };
struct uint4 { unsigned x, y, z, w; };
struct uint2 { unsigned x, y; };
inline uint2 make_uint2(unsigned a, unsigned b) { return {a, b}; }
struct float4 { float x, y, z, w; };
inline int4 make_int4(int a, int b, int c, int d) { return {a, b, c, d}; }
inline float4 make_float4(float a, float b, float c, float d) { return {a, b, c, d}; }
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return {a, b, c, d}; }
// per-halfword signed |x| (saturated) and signed maximum
inline unsigned __vabsss2(unsigned a)
{
    unsigned r = 0;
    for (int i = 0; i < 2; ++i) {
        const int h = (int16_t)(a >> (16 * i));
        r |= (unsigned)(uint16_t)(h == -32768 ? 32767 : (h < 0 ? -h : h)) << (16 * i);
    }
    return r;
}
inline unsigned __vmaxs2(unsigned a, unsigned b)
{
    unsigned r = 0;
    for (int i = 0; i < 2; ++i) {
        const int x = (int16_t)(a >> (16 * i)), y = (int16_t)(b >> (16 * i));
        r |= (unsigned)(uint16_t)(x > y ? x : y) << (16 * i);
    }
    return r;
}

inline int __clz(uint32_t x) { return x ? __builtin_clz(x) : 32; }
inline int __ffs(uint32_t x) { return x ? __builtin_ctz(x) + 1 : 0; }
inline int __ffs(int x) { return __ffs((uint32_t)x); }
inline float __int_as_float(int x) { float f; memcpy(&f, &x, 4); return f; }
inline float __uint_as_float(uint32_t x) { float f; memcpy(&f, &x, 4); return f; }
inline int __float_as_int(float f) { int x; memcpy(&x, &f, 4); return x; }
inline uint32_t __float_as_uint(float f) { uint32_t x; memcpy(&x, &f, 4); return x; }
inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned sh)
{
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (unsigned)(v >> (sh & 31));
}
inline unsigned __vcmpne4(unsigned a, unsigned b)
{
    unsigned r = 0;
    for (int i = 0; i < 4; ++i)
        if (((a >> (8 * i)) & 0xFF) != ((b >> (8 * i)) & 0xFF)) r |= 0xFFu << (8 * i);
    return r;
}
template <class T> inline T __ldcs(const T* p) { return *p; }
template <class T> inline T __ldg(const T* p) { return *p; }
template <class T> inline T __ldcg(const T* p) { return *p; }
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }

// block / warp synchronisation
void __syncthreads();
void __syncwarp(unsigned mask = 0xFFFFFFFFu);
unsigned __shfl_sync(unsigned mask, unsigned v, int src);
int __shfl_sync(unsigned mask, int v, int src);
int __shfl_up_sync(unsigned mask, int v, unsigned d);
int __shfl_down_sync(unsigned mask, int v, unsigned d);
unsigned __shfl_xor_sync(unsigned mask, unsigned v, int lanemask);
unsigned __ballot_sync(unsigned mask, int pred);
unsigned __reduce_and_sync(unsigned mask, unsigned v);
unsigned __reduce_max_sync(unsigned mask, unsigned v);
unsigned __reduce_add_sync(unsigned mask, unsigned v);
int __any_sync(unsigned mask, int pred);
// A warp vote is one convergence point per source site, as on the GPU: the
// host compiler may duplicate the call into divergent paths, so votes from
// kernel sources carry their file and line as the site instead of the
// return address.
unsigned emu_ballot_at(int pred, const char* file, int line);
#define __any_sync(mask, pred) (emu_ballot_at((pred), __FILE__, __LINE__) != 0u)
#define __ballot_sync(mask, pred) emu_ballot_at((pred), __FILE__, __LINE__)
unsigned char* emu_smem();
size_t emu_smem_bytes();
void emu_launch(unsigned blocks, unsigned threads, size_t smem, std::function<void()> body);
void emu_launch(const dim3& grid, unsigned threads, size_t smem, std::function<void()> body);

// CUDA runtime / driver stand-ins
typedef int cudaError_t;
constexpr int cudaSuccess = 0;
typedef void* cudaStream_t;
inline cudaError_t cudaGetLastError() { return 0; }
inline cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t) { memset(p, v, n); return 0; }

enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize };
template <class F> inline cudaError_t cudaFuncSetAttribute(F, cudaFuncAttribute, int) { return 0; }
struct cudaFuncAttributes { size_t sharedSizeBytes = 0; };
template <class F> inline cudaError_t cudaFuncGetAttributes(cudaFuncAttributes* a, F) { a->sharedSizeBytes = 0; return 0; }
template <class F> inline cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int* n, F, int, size_t) { *n = 2; return 0; }
typedef int cudaDriverEntryPointQueryResult;
constexpr int cudaDriverEntryPointSuccess = 0;
constexpr int cudaEnableDefault = 0;
typedef unsigned long long cuuint64_t;
typedef unsigned cuuint32_t;
typedef int CUresult;
constexpr int CUDA_SUCCESS = 0;
enum CUtensorMapDataType { CU_TENSOR_MAP_DATA_TYPE_INT32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32 };
enum CUtensorMapInterleave { CU_TENSOR_MAP_INTERLEAVE_NONE };
enum CUtensorMapSwizzle { CU_TENSOR_MAP_SWIZZLE_NONE };
enum CUtensorMapL2promotion { CU_TENSOR_MAP_L2_PROMOTION_NONE };
enum CUtensorMapFloatOOBfill { CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE };
struct CUtensorMap { char* base; unsigned long long dim0, dim1, stride; unsigned box0, box1; int valid; };
cudaError_t cudaGetDriverEntryPointByVersion(const char*, void** p, int, int, cudaDriverEntryPointQueryResult* q);
void emu_st_v8(void* q, int a0, int a1, int a2, int a3, int a4, int a5, int a6, int a7);
void emu_tma_store(const CUtensorMap* m, const void* buf, int x, int y);
void emu_bar_sync(int id, int n);
