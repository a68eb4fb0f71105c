// tt_misfit_noalloc: the misfit and adjoint sources of tt_misfit for callers that must not
// allocate device memory (see include/tt.h). Its scratch lives in one file-scope device
// array instead of a context's workspace.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tt.h"
#include "tt_aux.h"

using namespace ttgb;

namespace {

// Scratch layout: flags (256 B), receiver positions, receiver cell corners, weights.
constexpr size_t kFlagsBytes = 256;
constexpr size_t kRecOffset = kFlagsBytes;
constexpr size_t kCornerOffset = kRecOffset + sizeof(PointD) * TT_NOALLOC_MAX_REC;
constexpr size_t kWeightOffset = kCornerOffset + sizeof(long long) * 8 * TT_NOALLOC_MAX_REC;
constexpr size_t kScratchBytes = kWeightOffset + sizeof(double) * 8 * TT_NOALLOC_MAX_REC;
static_assert(kCornerOffset % 8 == 0 && kWeightOffset % 8 == 0, "scratch alignment");

}  // namespace

// Shared by every call on a device; held by each device that loads the library until exit.
static __device__ __align__(256) unsigned char g_misfit_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

void set_err(char *h_err, int err_len, const char *msg) {
    if (h_err && err_len > 0) {
        strncpy(h_err, msg, (size_t)err_len - 1);
        h_err[err_len - 1] = '\0';
    }
}

// Device address of the scratch array for the current device, looked up once per device.
unsigned char *scratch_address(int dev, char *h_err, int err_len) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_misfit_scratch);
        if (e != cudaSuccess) {
            char buf[160];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            set_err(h_err, err_len, buf);
            return nullptr;
        }
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    return g_scratch_ptr[dev];
}

bool point_inside(const tt_grid &G, const tt_point &p) {
    const double eps = 1e-9;
    double sd = G.depth_max_km - G.depth_min_km, st = G.lat_max_deg - G.lat_min_deg;
    double sp = G.lon_max_deg - G.lon_min_deg;
    return std::isfinite(p.depth_km) && std::isfinite(p.lat_deg) && std::isfinite(p.lon_deg) &&
           p.depth_km >= G.depth_min_km - eps * sd && p.depth_km <= G.depth_max_km + eps * sd &&
           p.lat_deg >= G.lat_min_deg - eps * st && p.lat_deg <= G.lat_max_deg + eps * st &&
           p.lon_deg >= G.lon_min_deg - eps * sp && p.lon_deg <= G.lon_max_deg + eps * sp;
}

}  // namespace

extern "C" tt_status tt_misfit_noalloc(const tt_grid *grid, const void *d_T, int dtype,
                                       const tt_data *d, double *d_Tr, double *d_chi,
                                       double *d_R, void *cuda_stream, char *h_err,
                                       int err_len) {
    GridC g;
    if (!grid || !grid_constants(*grid, g)) {
        set_err(h_err, err_len, "tt_misfit_noalloc: invalid grid");
        return TT_EINVAL;
    }
    if (!d || !d_T || !d_R || !d->d_abs_off || !d->d_cs_off || !d->h_rec) {
        set_err(h_err, err_len, "tt_misfit_noalloc: NULL argument");
        return TT_EINVAL;
    }
    if (dtype != TT_F32 && dtype != TT_F64) {
        set_err(h_err, err_len, "tt_misfit_noalloc: dtype is neither TT_F32 nor TT_F64");
        return TT_EINVAL;
    }
    if (d->n_src < 1 || d->n_src > TT_MAX_BATCH) {
        set_err(h_err, err_len, "tt_misfit_noalloc: n_src outside 1..TT_MAX_BATCH");
        return TT_EINVAL;
    }
    if (d->n_rec < 1 || d->n_rec > TT_NOALLOC_MAX_REC) {
        set_err(h_err, err_len,
                "tt_misfit_noalloc: n_rec must be 1..TT_NOALLOC_MAX_REC (the size of its "
                "static scratch); use tt_misfit for more receivers");
        return TT_EINVAL;
    }
    for (int m = 0; m < d->n_rec; ++m)
        if (!point_inside(*grid, d->h_rec[m])) {
            set_err(h_err, err_len, "tt_misfit_noalloc: receiver outside the grid");
            return TT_EINVAL;
        }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_err(h_err, err_len, "tt_misfit_noalloc: no usable current device");
        return TT_ECUDA;
    }
    unsigned char *base = scratch_address(dev, h_err, err_len);
    if (!base) return TT_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *flags = (int *)base;
    PointD *rec = (PointD *)(base + kRecOffset);
    long long *cq = (long long *)(base + kCornerOffset);
    double *wq = (double *)(base + kWeightOffset);

    cudaError_t e = cudaMemsetAsync(flags, 0, kFlagsBytes, st);  // flags must start at zero
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rec, d->h_rec, sizeof(PointD) * (size_t)d->n_rec,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = run_receiver_setup(g, rec, d->n_rec, cq, wq, flags + 1, st);
    if (e == cudaSuccess)
        e = dtype == TT_F32
                ? run_misfit<float>(d->n_src, d->n_rec, d_T, cq, wq, *d, d_Tr, d_chi, d_R, flags,
                                    st)
                : run_misfit<double>(d->n_src, d->n_rec, d_T, cq, wq, *d, d_Tr, d_chi, d_R, flags,
                                     st);
    int h_flags[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_flags, flags, sizeof h_flags, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "tt_misfit_noalloc: %s", cudaGetErrorString(e));
        set_err(h_err, err_len, buf);
        return TT_ECUDA;
    }
    if (h_flags[0]) {
        set_err(h_err, err_len, "tt_misfit_noalloc: receiver index out of range in the data");
        return TT_EINVAL;
    }
    if (h_flags[1]) {
        set_err(h_err, err_len, "tt_misfit_noalloc: receiver outside the grid");
        return TT_EINVAL;
    }
    set_err(h_err, err_len, "");
    return TT_OK;
}
