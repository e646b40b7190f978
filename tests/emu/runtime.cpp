// Runtime of the host emulation of libedt's kernels (test infrastructure).
//
// Every CUDA thread of a block is a user-space fiber (ucontext); the blocks
// of a launch run one after the other on one OS thread.  __syncthreads, named
// barriers and every warp collective (shuffle, ballot, vote, reduce,
// __syncwarp) make the fiber yield; a barrier is released when every fiber
// it concerns has arrived.  A warp collective that the 32 lanes of a warp
// reach from different call sites, or that some lane never reaches, aborts
// with a message (on a GPU that would be undefined behaviour or a hang).
// Dynamic shared memory is one malloc of exactly the requested size, so that
// AddressSanitizer reports any access past it; global memory is host memory.
// TMA tile stores and 32-byte vector stores are carried out in C++ with the
// hardware's alignment and bounds rules checked.
#include "shim.h"
// the runtime defines the votes themselves (the shim's macros are for kernel sources)
#undef __any_sync
#undef __ballot_sync
#include <ucontext.h>
#include <sanitizer/common_interface_defs.h>

struct Fiber {
    ucontext_t ctx;
    char* stack;
    size_t stack_size;
    int tid;
    int state;   // 0 runnable, 1 at block barrier, 2 at warp barrier, 3 at named barrier, 4 done
    int named;
    const void* tag;
    void* fake_stack;
};
static std::vector<Fiber> g_f;
static ucontext_t g_main;
static int g_cur = -1;
static unsigned char* g_smem = nullptr;
static size_t g_smem_bytes = 0;
static std::function<void()> g_body;
static unsigned g_block, g_blocks, g_threads, g_gridx = 0;
static uint32_t g_slot[32][32];   // [warp][lane]
thread_local EmuDim threadIdx, blockIdx, blockDim, gridDim;
static const void* g_main_stack_bottom; static size_t g_main_stack_size;

static void set_ids(int t)
{
    threadIdx.x = t;
    blockDim.x = g_threads;
    if (g_gridx) {
        blockIdx.x = g_block % g_gridx;
        blockIdx.y = g_block / g_gridx;
        gridDim.x = g_gridx;
        gridDim.y = g_blocks / g_gridx;
    } else {
        blockIdx.x = g_block;
        blockIdx.y = 0;
        gridDim.x = g_blocks;
        gridDim.y = 1;
    }
}

static void yield_to_main()
{
    Fiber& f = g_f[g_cur];
    __sanitizer_start_switch_fiber(&f.fake_stack, g_main_stack_bottom, g_main_stack_size);
    swapcontext(&f.ctx, &g_main);
    __sanitizer_finish_switch_fiber(f.fake_stack, nullptr, nullptr);
    set_ids(g_f[g_cur].tid);
}
static void fiber_entry()
{
    __sanitizer_finish_switch_fiber(nullptr, &g_main_stack_bottom, &g_main_stack_size);
    set_ids(g_f[g_cur].tid);
    g_body();
    g_f[g_cur].state = 4;
    Fiber& f = g_f[g_cur];
    __sanitizer_start_switch_fiber(nullptr, g_main_stack_bottom, g_main_stack_size);
    swapcontext(&f.ctx, &g_main);
}

void __syncthreads() { g_f[g_cur].state = 1; yield_to_main(); }
static void warp_wait(const void* tag) { g_f[g_cur].state = 2; g_f[g_cur].tag = tag; yield_to_main(); }
void __syncwarp(unsigned) { warp_wait(__builtin_return_address(0)); }
void emu_bar_sync(int id, int n) { g_f[g_cur].state = 3; g_f[g_cur].named = id * 4096 + n; yield_to_main(); }
static uint32_t xchg(uint32_t v, int src, const void* tag)
{
    const int t = g_f[g_cur].tid;
    g_slot[t >> 5][t & 31] = v;
    warp_wait(tag);
    const uint32_t r = g_slot[t >> 5][src & 31];
    warp_wait(tag);
    return r;
}
unsigned __shfl_sync(unsigned, unsigned v, int src) { return xchg(v, src, __builtin_return_address(0)); }
int __shfl_sync(unsigned, int v, int src) { return (int)xchg((uint32_t)v, src, __builtin_return_address(0)); }
unsigned __shfl_xor_sync(unsigned, unsigned v, int lanemask)
{
    const int lane = g_f[g_cur].tid & 31;
    return xchg(v, lane ^ (lanemask & 31), __builtin_return_address(0));
}
int __shfl_up_sync(unsigned, int v, unsigned d)
{
    const int lane = g_f[g_cur].tid & 31;
    const int src = lane >= (int)d ? lane - (int)d : lane;
    return (int)xchg((uint32_t)v, src, __builtin_return_address(0));
}
int __shfl_down_sync(unsigned, int v, unsigned d)
{
    const int lane = g_f[g_cur].tid & 31;
    const int src = lane + (int)d < 32 ? lane + (int)d : lane;
    return (int)xchg((uint32_t)v, src, __builtin_return_address(0));
}
static unsigned ballot_tag(int pred, const void* tag)
{
    const int t = g_f[g_cur].tid;
    g_slot[t >> 5][t & 31] = pred ? 1u : 0u;
    warp_wait(tag);
    unsigned r = 0;
    for (int l = 0; l < 32; ++l) r |= g_slot[t >> 5][l] << l;
    warp_wait(tag);
    return r;
}
unsigned __ballot_sync(unsigned, int pred) { return ballot_tag(pred, __builtin_return_address(0)); }
int __any_sync(unsigned, int pred) { return ballot_tag(pred, __builtin_return_address(0)) != 0; }
unsigned emu_ballot_at(int pred, const char* file, int line)
{
    // a site tag from the file name's address and the line
    return ballot_tag(pred, reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(file) * 65599u + (uintptr_t)line));
}
unsigned __reduce_and_sync(unsigned, unsigned v)
{
    const int t = g_f[g_cur].tid;
    g_slot[t >> 5][t & 31] = v;
    warp_wait(__builtin_return_address(0));
    unsigned r = 0xFFFFFFFFu;
    for (int l = 0; l < 32; ++l) r &= g_slot[t >> 5][l];
    warp_wait(__builtin_return_address(0));
    return r;
}
unsigned __reduce_max_sync(unsigned, unsigned v)
{
    const int t = g_f[g_cur].tid;
    g_slot[t >> 5][t & 31] = v;
    warp_wait(__builtin_return_address(0));
    unsigned r = 0u;
    for (int l = 0; l < 32; ++l) r = g_slot[t >> 5][l] > r ? g_slot[t >> 5][l] : r;
    warp_wait(__builtin_return_address(0));
    return r;
}
unsigned __reduce_add_sync(unsigned, unsigned v)
{
    const int t = g_f[g_cur].tid;
    g_slot[t >> 5][t & 31] = v;
    warp_wait(__builtin_return_address(0));
    unsigned r = 0u;
    for (int l = 0; l < 32; ++l) r += g_slot[t >> 5][l];
    warp_wait(__builtin_return_address(0));
    return r;
}
unsigned char* emu_smem() { return g_smem; }
size_t emu_smem_bytes() { return g_smem_bytes; }

static void launch_blocks(unsigned blocks, unsigned threads, size_t smem, std::function<void()> body);
void emu_launch(unsigned blocks, unsigned threads, size_t smem, std::function<void()> body)
{
    g_gridx = 0;
    launch_blocks(blocks, threads, smem, body);
}
void emu_launch(const dim3& grid, unsigned threads, size_t smem, std::function<void()> body)
{
    g_gridx = grid.x;
    launch_blocks(grid.x * grid.y, threads, smem, body);
    g_gridx = 0;
}
static void launch_blocks(unsigned blocks, unsigned threads, size_t smem, std::function<void()> body)
{
    if (threads % 32 != 0 || threads == 0 || threads > 1024) { fprintf(stderr, "bad block size %u\n", threads); abort(); }
    if (smem > 227 * 1024) { fprintf(stderr, "smem %zu too large\n", smem); abort(); }
    g_body = body;
    g_blocks = blocks;
    g_threads = threads;
    const size_t SS = 256 * 1024;
    g_f.assign(threads, Fiber{});
    for (unsigned t = 0; t < threads; ++t) { g_f[t].stack = (char*)malloc(SS); g_f[t].stack_size = SS; }
    for (unsigned b = 0; b < blocks; ++b) {
        g_block = b;
        g_smem = smem ? (unsigned char*)malloc(smem) : nullptr;
        if (g_smem) memset(g_smem, 0xCD, smem);
        g_smem_bytes = smem;
        for (unsigned t = 0; t < threads; ++t) {
            Fiber& f = g_f[t];
            f.tid = t; f.state = 0; f.fake_stack = nullptr;
            getcontext(&f.ctx);
            f.ctx.uc_stack.ss_sp = f.stack;
            f.ctx.uc_stack.ss_size = f.stack_size;
            f.ctx.uc_link = nullptr;
            makecontext(&f.ctx, fiber_entry, 0);
        }
        for (;;) {
            bool ran = false;
            for (unsigned t = 0; t < threads; ++t) {
                if (g_f[t].state != 0) continue;
                g_cur = t;
                void* fs = nullptr;
                __sanitizer_start_switch_fiber(&fs, g_f[t].stack, g_f[t].stack_size);
                swapcontext(&g_main, &g_f[t].ctx);
                __sanitizer_finish_switch_fiber(fs, nullptr, nullptr);
                ran = true;
            }
            if (ran) continue;
            // release barriers
            bool alldone = true, released = false;
            for (auto& f : g_f) alldone &= f.state == 4;
            if (alldone) break;
            // warp barriers: all 32 lanes at state 2
            for (unsigned w = 0; w < threads / 32; ++w) {
                bool all = true;
                for (int l = 0; l < 32; ++l) all &= g_f[w * 32 + l].state == 2;
                if (all) for (int l = 1; l < 32; ++l)
                    if (g_f[w * 32 + l].tag != g_f[w * 32].tag) { fprintf(stderr, "divergent warp collective: warp %u lanes 0 and %d at different sites\n", w, l); abort(); }
                if (all) { for (int l = 0; l < 32; ++l) g_f[w * 32 + l].state = 0; released = true; }
            }
            if (released) continue;
            // block barrier: every live fiber at state 1
            bool all1 = true; int live = 0;
            for (auto& f : g_f) if (f.state != 4) { ++live; all1 &= f.state == 1; }
            if (all1 && live > 0) {
                for (auto& f : g_f) if (f.state == 1) f.state = 0;
                continue;
            }
            // named barriers
            std::vector<int> cnt(64 * 4096 + 1, 0);
            for (auto& f : g_f) if (f.state == 3) cnt[f.named]++;
            for (auto& f : g_f) if (f.state == 3 && cnt[f.named] == (f.named & 4095)) { f.state = 0; released = true; }
            if (released) continue;
            fprintf(stderr, "emulator deadlock in block %u\n", b);
            for (auto& f : g_f) fprintf(stderr, " t%d:%d", f.tid, f.state);
            fprintf(stderr, "\n");
            abort();
        }
        free(g_smem);
        g_smem = nullptr;
    }
    for (auto& f : g_f) free(f.stack);
    g_f.clear();
}
void emu_st_v8(void* q, int a0, int a1, int a2, int a3, int a4, int a5, int a6, int a7)
{
    if (reinterpret_cast<uintptr_t>(q) & 31) { fprintf(stderr, "st_v8 misaligned %p\n", q); abort(); }
    int* p = (int*)q;
    p[0] = a0; p[1] = a1; p[2] = a2; p[3] = a3; p[4] = a4; p[5] = a5; p[6] = a6; p[7] = a7;
}

void emu_tma_store(const CUtensorMap* m, const void* buf, int x, int y)
{
    if (!m->valid) { fprintf(stderr, "tma store with invalid map\n"); abort(); }
    if ((x * 4) % 16 != 0 || x < 0 || y < 0) { fprintf(stderr, "tma store bad coords x=%d y=%d\n", x, y); abort(); }
    if ((unsigned long long)x >= m->dim0 || (unsigned long long)y >= m->dim1) { fprintf(stderr, "tma box starts outside x=%d y=%d\n", x, y); abort(); }
    const unsigned char* sb = (const unsigned char*)buf;
    if (!(sb >= g_smem && sb + m->box0 * m->box1 * 4 <= g_smem + g_smem_bytes)) { fprintf(stderr, "tma staging outside smem\n"); abort(); }
    if ((uintptr_t)(sb - g_smem) % 16) { fprintf(stderr, "tma staging not 16-aligned\n"); abort(); }
    const int* s = (const int*)buf;
    for (unsigned r = 0; r < m->box1; ++r)
        for (unsigned c = 0; c < m->box0; ++c) {
            const unsigned long long gx = x + c, gy = y + r;
            if (gx < m->dim0 && gy < m->dim1)
                memcpy(m->base + gy * m->stride + gx * 4, &s[r * m->box0 + c], 4);
        }
}

static CUresult fake_encode(CUtensorMap* m, CUtensorMapDataType, cuuint32_t rank, void* base, const cuuint64_t* dims,
                            const cuuint64_t* strides, const cuuint32_t* box, const cuuint32_t*, CUtensorMapInterleave,
                            CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill)
{
    if (rank != 2 || (reinterpret_cast<uintptr_t>(base) & 15) || strides[0] % 16) return 1;
    m->base = (char*)base; m->dim0 = dims[0]; m->dim1 = dims[1]; m->stride = strides[0];
    m->box0 = box[0]; m->box1 = box[1]; m->valid = 1;
    return 0;
}
cudaError_t cudaGetDriverEntryPointByVersion(const char*, void** p, int, int, cudaDriverEntryPointQueryResult* q)
{
    *p = (void*)&fake_encode;
    *q = 0;
    return 0;
}

// libedt's kernel tracing lives in its API file, which the emulation does
// not build: tracing is off here.
namespace edt {
bool trace_on() { return false; }
int trace_begin(const char*, cudaStream_t) { return 0; }
void trace_end(int, cudaStream_t) {}
}  // namespace edt
