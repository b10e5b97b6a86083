// Line smoothing without any device allocation.
//
// ellsolve_level_smooth allocates a partner buffer and Thomas scratch with
// cudaMalloc on every call.  Some callers cannot do that: a host program that
// hands the library a fixed device-memory budget owned by its own allocator or
// memory pool (a cudaMalloc behind the pool's back would overrun the budget or
// fail once the pool holds the memory), and latency-critical loops where a
// cudaMalloc / cudaFree pair may synchronise the device or fragment memory.
// ellsolve_level_smooth_noalloc runs the same kernels with all of its scratch
// -- the level descriptor, the work items, the partner iterate and the Thomas
// scratch -- carved out of one file-scope device array of kStaticScratchBytes.
// It copies the descriptor and items from host memory and waits for its
// stream before returning, so it is an ordinary blocking call.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "ellsolve.h"
#include "kernels.hpp"
#include "solver.hpp"

namespace {

using namespace ells;

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB on every device that loads us

// Device-side array: host code may only use its address as returned by
// cudaGetSymbolAddress (the host symbol itself is a stand-in, not device memory).
static __device__ __align__(256) unsigned char g_smooth_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
std::vector<void *> g_addr;  // device address of g_smooth_scratch, per device ordinal

// Address of the scratch array on the current device, looked up once per device.
void *scratch_on_current_device() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (int(g_addr.size()) <= dev) g_addr.resize(dev + 1, nullptr);
    if (!g_addr[dev]) {
        void *p = nullptr;
        check_cuda(cudaGetSymbolAddress(&p, g_smooth_scratch), "cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
ellsolve_status smooth_static(Problem &p, int level, const void *b, void *u, int nsweeps,
                              double rho) {
    if (level < 0 || level >= p.nlev) throw Error(ELLSOLVE_ERR_ARG, "level out of range");
    // the scratch array is per device: the handle's buffers and stream live on
    // the device current at its creation, so the same device must be current
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p.device)
        throw Error(ELLSOLVE_ERR_ARG, "current device " + std::to_string(dev) +
                                          " is not the handle's device " + std::to_string(p.device));
    if (sizeof(T) == 8 && level > 0 && p.opts.precision != 0)
        throw Error(ELLSOLVE_ERR_ARG, "FP64 coarse levels exist only with precision 0");
    if (sizeof(T) == 4 && p.opts.precision != 1)
        throw Error(ELLSOLVE_ERR_ARG, "FP32 levels exist only with precision 1");
    const LevelStore &Ls = p.lev[level];
    const size_t nl = size_t(Ls.ncol) * p.nz;
    const int per = div_up(Ls.ncol, kBlk);
    // layout: [descriptor][items: even sweeps, odd sweeps][partner iterate][Thomas scratch]
    const size_t off_items = round_up(sizeof(Lv<T>), 256);
    const size_t off_part = round_up(off_items + size_t(2) * per * sizeof(Item), 256);
    const size_t off_aux = round_up(off_part + nl * sizeof(T), 256);
    const size_t need = off_aux + nl * sizeof(T);
    if (need > kStaticScratchBytes)
        throw Error(ELLSOLVE_ERR_CAPACITY,
                    "level needs " + std::to_string(need) + " bytes of scratch; the static array "
                    "holds " + std::to_string(kStaticScratchBytes));
    unsigned char *base = static_cast<unsigned char *>(scratch_on_current_device());

    Lv<T> d;
    if (sizeof(T) == 8) std::memcpy(&d, &p.h64[level], sizeof(d));
    else std::memcpy(&d, &p.h32[level], sizeof(d));
    d.b = static_cast<T *>(const_cast<void *>(b));
    d.u[0] = static_cast<T *>(u);
    d.u[1] = reinterpret_cast<T *>(base + off_part);
    d.aux = reinterpret_cast<T *>(base + off_aux);
    // block red-black SOR: a sweep is two half-sweeps, red from the iterate
    // into the partner buffer, then black back (the parity fixes the colour)
    const bool rb = p.opts.smoother == 1;
    std::vector<Item> items(size_t(2) * per);
    for (int parity = 0; parity < 2; ++parity)
        for (int i = 0; i < per; ++i) {
            Item &it = items[size_t(parity) * per + i];
            it.lv = 0;
            it.col0 = i * kBlk;
            it.in = (unsigned char)parity;
            it.out = (unsigned char)(1 - parity);
            it.zero = 0;
            it.colour = (unsigned char)(rb ? parity + 1 : 0);
        }
    cudaStream_t s = p.stream;
    // pageable sources: the CUDA driver stages the copies, nothing is allocated here
    check_cuda(cudaMemcpyAsync(base, &d, sizeof(d), cudaMemcpyHostToDevice, s), "descriptor");
    check_cuda(cudaMemcpyAsync(base + off_items, items.data(), items.size() * sizeof(Item),
                               cudaMemcpyHostToDevice, s),
               "items");
    const Lv<T> *L = reinterpret_cast<const Lv<T> *>(base);
    const Item *it = reinterpret_cast<const Item *>(base + off_items);
    const bool rows = sizeof(T) == 4 && rows_eligible(p, level);
    const int launches = rb ? 2 * nsweeps : nsweeps;
    for (int sw = 0; sw < launches; ++sw)
        launch_smoother<T>(p, s, L, it + size_t(sw & 1) * per, per, rho, p.nz, 0, rows,
                           p.lev[level].n % 32 == 0, level);
    if (launches & 1)
        check_cuda(cudaMemcpyAsync(u, d.u[1], nl * sizeof(T), cudaMemcpyDeviceToDevice, s),
                   "copy back");
    check_cuda(cudaStreamSynchronize(s), "noalloc sync");
    return ELLSOLVE_OK;
}

}  // namespace

extern "C" ellsolve_status ellsolve_level_smooth_noalloc(ellsolve_t h, int level, int fp32,
                                                         const void *b, void *u, int nsweeps,
                                                         double rho) {
    try {
        if (!h || !b || !u || nsweeps < 0) throw Error(ELLSOLVE_ERR_ARG, "bad argument");
        if (nsweeps == 0) return ELLSOLVE_OK;
        Problem &p = *h;
        return fp32 ? smooth_static<float>(p, level, b, u, nsweeps, rho)
                    : smooth_static<double>(p, level, b, u, nsweeps, rho);
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return ELLSOLVE_ERR_ARG;
    }
}
