// api.cu -- library and context entry points of libblsh (version, errors,
// context creation, blsh_status).
#include <stdarg.h>

#include "common.cuh"

int blsh_fail(blsh_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int blsh_cuda_check(blsh_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BLSH_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return blsh_fail(ctx, BLSH_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return blsh_fail(ctx, BLSH_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *blsh_version(void) { return "libblsh 0.1 (sm_103a)"; }

extern "C" const char *blsh_strerror(int code) {
    switch (code) {
    case BLSH_OK: return "ok";
    case BLSH_EINVAL: return "invalid argument";
    case BLSH_ERANGE: return "pair index out of range";
    case BLSH_ETRUNC: return "output truncated";
    case BLSH_ENOMEM: return "out of memory";
    case BLSH_EDEVICE: return "CUDA error";
    case BLSH_ENUMERIC: return "numerical problem in the inference tables";
    case BLSH_ESIZE: return "problem larger than a fixed-size scratch array of the library";
    default: return "unknown error";
    }
}

extern "C" int blsh_ctx_create(blsh_ctx **out, int device) {
    if (!out) return BLSH_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return BLSH_EDEVICE;
    }
    blsh_ctx *ctx = new blsh_ctx();
    ctx->device = device;
    blsh_device_guard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return BLSH_EDEVICE;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->cc_major = prop.major;
    ctx->cc_minor = prop.minor;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (prop.major != 10 || prop.minor != 3) {
        // The kernels are compiled for sm_103a only.
        delete ctx;
        return BLSH_EDEVICE;
    }
    if (cudaMalloc((void **)&ctx->scratch, sizeof(blsh_dev_scratch)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return BLSH_ENOMEM;
    }
    if (cudaMalloc((void **)&ctx->recheck_queue, sizeof(uint2) * BLSH_RECHECK_CAP) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->scratch);
        delete ctx;
        return BLSH_ENOMEM;
    }
    if (cudaMalloc((void **)&ctx->lite_queue, sizeof(unsigned long long) * BLSH_LITE_QUEUE_CAP) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->scratch);
        cudaFree(ctx->recheck_queue);
        delete ctx;
        return BLSH_ENOMEM;
    }
    if (cudaMemset(ctx->scratch, 0, sizeof(blsh_dev_scratch)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(ctx->scratch);
        cudaFree(ctx->recheck_queue);
        cudaFree(ctx->lite_queue);
        delete ctx;
        return BLSH_EDEVICE;
    }
    *out = ctx;
    return BLSH_OK;
}

static void timing_release(blsh_ctx *ctx);

extern "C" int blsh_ctx_destroy(blsh_ctx *ctx) {
    if (!ctx) return BLSH_OK;
    {
        blsh_device_guard g(ctx->device);
        timing_release(ctx);
        if (ctx->plane) cudaFree(ctx->plane);
        if (ctx->norm2) cudaFree(ctx->norm2);
        if (ctx->scratch) cudaFree(ctx->scratch);
        if (ctx->recheck_queue) cudaFree(ctx->recheck_queue);
        if (ctx->lite_queue) cudaFree(ctx->lite_queue);
    }
    delete ctx;
    return BLSH_OK;
}

extern "C" int blsh_ctx_reserve(blsh_ctx *ctx, int64_t max_objects) {
    if (!ctx) return BLSH_EINVAL;
    if (max_objects < 0 || max_objects > (1ll << 32)) return blsh_fail(ctx, BLSH_EINVAL, "max_objects outside 0..2^32");
    if (max_objects > 0 && max_objects <= ctx->plane_cap && max_objects <= ctx->norm2_cap) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    // work already enqueued may still read the old buffers
    BLSH_CUDA(ctx, cudaDeviceSynchronize());
    if (ctx->plane) BLSH_CUDA(ctx, cudaFree(ctx->plane));
    if (ctx->norm2) BLSH_CUDA(ctx, cudaFree(ctx->norm2));
    ctx->plane = ctx->norm2 = nullptr;
    ctx->plane_cap = ctx->norm2_cap = 0;
    if (max_objects == 0) return BLSH_OK;
    BLSH_CUDA(ctx, cudaMalloc(&ctx->plane, (size_t)max_objects * sizeof(uint4)));
    const cudaError_t e = cudaMalloc(&ctx->norm2, (size_t)max_objects * sizeof(long long));
    if (e != cudaSuccess) {
        cudaFree(ctx->plane);
        ctx->plane = nullptr;
        return blsh_cuda_check(ctx, e, "cudaMalloc(norm2)");
    }
    ctx->plane_cap = ctx->norm2_cap = max_objects;
    return BLSH_OK;
}

extern "C" int64_t blsh_ctx_reserved(const blsh_ctx *ctx) {
    if (!ctx) return -1;
    return ctx->plane_cap < ctx->norm2_cap ? ctx->plane_cap : ctx->norm2_cap;
}

extern "C" const char *blsh_last_error(const blsh_ctx *ctx) { return ctx ? ctx->err : "no context"; }

extern "C" int blsh_status(blsh_ctx *ctx, void *stream, uint64_t *counters) {
    if (!ctx) return BLSH_EINVAL;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return blsh_cuda_check(ctx, e, "cudaStreamSynchronize");
    struct {
        unsigned int err_code, pad0;
        unsigned long long counters[4];
    } h;
    BLSH_CUDA(ctx, cudaMemcpyAsync(&h, ctx->scratch, sizeof(h), cudaMemcpyDeviceToHost, s));
    BLSH_CUDA(ctx, cudaMemsetAsync(ctx->scratch, 0, sizeof(h), s));
    BLSH_CUDA(ctx, cudaStreamSynchronize(s));
    if (counters)
        for (int i = 0; i < 4; i++) counters[i] = h.counters[i];
    if (h.err_code == BLSH_ERANGE)
        return blsh_fail(ctx, BLSH_ERANGE, "%llu pairs named an object index >= N", h.counters[0]);
    if (h.err_code == BLSH_ETRUNC)
        return blsh_fail(ctx, BLSH_ETRUNC, "%llu outputs exceeded their capacity", h.counters[1]);
    if (h.err_code != 0) return blsh_fail(ctx, (int)h.err_code, "device error %u", h.err_code);
    return BLSH_OK;
}

extern "C" int64_t blsh_launch_count(const blsh_ctx *ctx) {
    return ctx ? (int64_t)ctx->launches.load(std::memory_order_relaxed) : -1;
}

static void timing_release(blsh_ctx *ctx) {
    auto &T = ctx->timing;
    for (cudaEvent_t e : T.ev)
        if (e) cudaEventDestroy(e);
    T.ev.clear();
    T.name.clear();
    T.on = T.open = false;
    T.cap = T.n = 0;
}

extern "C" int blsh_timing_begin(blsh_ctx *ctx, int32_t max_launches) {
    if (!ctx) return BLSH_EINVAL;
    if (max_launches <= 0 || max_launches > 65536) return blsh_fail(ctx, BLSH_EINVAL, "max_launches outside 1..65536");
    blsh_device_guard g(ctx->device);
    timing_release(ctx);
    auto &T = ctx->timing;
    T.ev.assign(2 * (size_t)max_launches, nullptr);
    T.name.assign((size_t)max_launches, nullptr);
    for (auto &e : T.ev) {
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            e = nullptr;
            timing_release(ctx);
            return blsh_cuda_check(ctx, r, "cudaEventCreate");
        }
    }
    T.cap = max_launches;
    T.on = true;
    return BLSH_OK;
}

extern "C" int blsh_timing_end(blsh_ctx *ctx, int32_t max, const char **names, float *ms, int32_t *n) {
    if (!ctx) return BLSH_EINVAL;
    if (max < 0 || (max > 0 && (!names || !ms)) || !n) return blsh_fail(ctx, BLSH_EINVAL, "bad output arrays");
    blsh_device_guard g(ctx->device);
    auto &T = ctx->timing;
    int out = 0, rc = BLSH_OK;
    for (int i = 0; i < T.n && out < max; ++i) {
        cudaError_t e = cudaEventSynchronize(T.ev[2 * i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, T.ev[2 * i], T.ev[2 * i + 1]);
        if (e != cudaSuccess) {
            rc = blsh_cuda_check(ctx, e, "cudaEventElapsedTime");
            break;
        }
        names[out] = T.name[i];
        ms[out++] = t;
    }
    *n = out;
    timing_release(ctx);
    return rc;
}
