// An entry point that allocates no device memory: one MUSCL-HLLC explicit
// Euler step in FP32 on caller-owned device buffers.
//
// Who needs it: code that must not call cudaMalloc or any allocator -- for
// example a plug-in that runs inside a host application whose memory pools
// own the device (or that runs while such an application forbids allocation
// in its hot loop), or a real-time loop where an allocation could block.
// Such a caller owns its inputs and outputs; the only scratch this step needs
// (the face values of the wet cells, 48 bytes per cell, plus a few scalars)
// lives in the fixed array below, compiled into the library.
//
// Limits and sharing rules:
//  - at most SWE_NOALLOC_MAX_CELLS cells per call (a larger mesh is rejected);
//  - the array exists once per GPU that loads the library and stays allocated
//    until the process exits;
//  - every call on a GPU uses the same array: calls that overlap on the GPU
//    (other streams, other threads) race on it and give wrong results;
//  - the first call on each GPU looks up the array's device address with
//    cudaGetSymbolAddress (with that GPU current); make that first call
//    before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "swe_dev.h"

void swe_set_error(const std::string &msg);

namespace {

constexpr size_t kFaceBytes = (size_t)SWE_NOALLOC_MAX_CELLS * 3 * sizeof(Vec4<float>);
constexpr size_t kScalarOff = kFaceBytes;                               // DevScalars
constexpr size_t kDtOff = kScalarOff + 256;                             // the step's dt (one double)
constexpr size_t kHistOff = kDtOff + 256;                               // dt history ring
constexpr size_t kScratchBytes = kHistOff + SWE_DT_HISTORY * sizeof(double);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current GPU (set up once per GPU).
int scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        swe_set_error(std::string("swe_muscl_step_noalloc: no current GPU: ") + cudaGetErrorString(e));
        return SWE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            swe_set_error(std::string("swe_muscl_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return SWE_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return SWE_OK;
}

// Clears the step's scalars that the previous call left and stores this
// call's dt, both in the scratch array; dt arrives by value as a kernel
// argument, so nothing is copied from host memory.
__global__ void k_noalloc_reset(DevScalars *sc, double *dtv, double dt)
{
    if (threadIdx.x == 0) {
        *sc = DevScalars{};
        *dtv = dt;
    }
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    if (!a || !b) return false;
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" int swe_muscl_step_noalloc(int64_t n_cells, const int32_t *nbr, const float *ln, const float *z,
                                      const float *manning_n, const float *h, const float *hu,
                                      const float *hv, float *h_out, float *hu_out, float *hv_out, double dt,
                                      const swe_params *p, const float *inflow_qlen, int n_inflow,
                                      const float *level, int n_level, void *stream)
{
    if (n_cells <= 0 || n_cells > SWE_NOALLOC_MAX_CELLS) {
        swe_set_error("swe_muscl_step_noalloc: n_cells must be in 1.." + std::to_string(SWE_NOALLOC_MAX_CELLS) +
                      ", got " + std::to_string(n_cells));
        return SWE_ERR_ARG;
    }
    if (!nbr || !ln || !z || !h || !hu || !hv || !h_out || !hu_out || !hv_out || !p ||
        !(dt >= 0.0) || !std::isfinite(dt) || p->precision != SWE_FP32 || p->scheme != SWE_SCHEME_MUSCL ||
        p->hr_order != 1 || !(p->g > 0) || !(p->h_eps > 0) || n_inflow < 0 || n_inflow > SWE_MAX_GROUPS ||
        n_level < 0 || n_level > SWE_MAX_GROUPS || (n_inflow > 0 && !inflow_qlen) || (n_level > 0 && !level) ||
        p->block < 0 || p->block > 1024 || (p->block % 32) != 0) {
        swe_set_error("swe_muscl_step_noalloc: bad argument (null pointer, non-finite or negative dt, "
                      "or params other than FP32 MUSCL with hr_order 1)");
        return SWE_ERR_ARG;
    }
    // every output must be apart from every other output and from every input
    {
        const size_t nf = (size_t)n_cells * sizeof(float);
        const void *outs[3] = {h_out, hu_out, hv_out};
        const void *ins[7] = {h, hu, hv, z, manning_n, ln, nbr};
        const size_t in_len[7] = {nf, nf, nf, nf, nf, 6 * nf, 3 * (size_t)n_cells * sizeof(int32_t)};
        bool bad = overlaps(outs[0], nf, outs[1], nf) || overlaps(outs[0], nf, outs[2], nf) ||
                   overlaps(outs[1], nf, outs[2], nf);
        for (int o = 0; o < 3 && !bad; o++)
            for (int q = 0; q < 7 && !bad; q++) bad = overlaps(outs[o], nf, ins[q], in_len[q]);
        if (bad) {
            swe_set_error("swe_muscl_step_noalloc: an output overlaps another output or an input");
            return SWE_ERR_ARG;
        }
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SWE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Vec4<float> *F = reinterpret_cast<Vec4<float> *>(base);
    DevScalars *sc = reinterpret_cast<DevScalars *>(base + kScalarOff);
    double *dtv = reinterpret_cast<double *>(base + kDtOff);
    // the scalars keep the previous call's values: clear them and set dt
    // (one small kernel on the stream; dt travels as its argument)
    k_noalloc_reset<<<1, 32, 0, st>>>(sc, dtv, dt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        swe_set_error(std::string("swe_muscl_step_noalloc: ") + cudaGetErrorString(e));
        return SWE_ERR_CUDA;
    }
    StepArgs<float> a{};
    a.m.n = n_cells;
    a.m.nbr = nbr;
    a.m.ln = reinterpret_cast<const Vec2<float> *>(ln);
    a.m.dd = nullptr;   // MUSCL derives the centroid offsets from ln
    a.m.z = z;
    a.m.nman = manning_n;
    a.m.area = nullptr;
    a.h = h; a.hu = hu; a.hv = hv;
    a.ho = h_out; a.huo = hu_out; a.hvo = hv_out;
    a.F = F; a.U = nullptr;
    a.sc = sc;
    a.dtv = dtv;
    a.dt_hist = reinterpret_cast<double *>(base + kHistOff);
    a.slot_cur = 0; a.slot_next = 1; a.slot_clear = 2;
    a.mode = MODE_EULER;
    a.cfl_rmin = 0.0;
    a.g = (float)p->g; a.h_eps = (float)p->h_eps; a.r_eps = (float)p->r_eps;
    a.waf_limiter = p->waf_limiter;
    for (int g = 0; g < n_inflow; g++) a.qlen[g] = inflow_qlen[g];
    for (int g = 0; g < n_level; g++) a.level[g] = level[g];
    const int block = p->block > 0 ? p->block : 256;
    e = launch_prep<float>(SWE_SCHEME_MUSCL, a, F, nullptr, block, st);
    if (e == cudaSuccess) e = launch_flux<float>(SWE_SCHEME_MUSCL, a, block, st);
    if (e != cudaSuccess) {
        swe_set_error(std::string("swe_muscl_step_noalloc: launch failed: ") + cudaGetErrorString(e));
        return SWE_ERR_CUDA;
    }
    return SWE_OK;
}
