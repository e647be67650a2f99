// lbs_internal.h — library-internal declarations shared by the single-instance
// API (lbs_api.cu) and the batched sweep (lbs_batch.cu): the context, the
// per-instance solver interface and its factory.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "../../include/lbs.h"

namespace lbs {

// one solver instance (Solver<R, P> in lbs_api.cu)
struct Base {
    virtual ~Base() {}
    virtual int init(const double *, const double *, const double *, const double *) = 0;
    virtual int step(int n) = 0;
    virtual int sync() = 0;
    virtual int get(double *, double *, double *, double *, double *) = 0;
    virtual int diag(lbs_diag *) = 0;
    virtual int profile(int on) = 0;
    virtual int kernel_times(double *ms, int n) = 0;
    virtual int kernel_count() const = 0;
    virtual int set_graph(int on) = 0;
    virtual int macro(double *, double *, double *, double *, double *, double *) = 0;
    // host copy of the device descriptor Inst<R> of this instance, and its size
    virtual const void *inst() const = 0;
    virtual size_t inst_bytes() const = 0;
    // member of a batch (2D): the batch runs the per-cell kernels, which keep
    // populations and moments in set 0 and start the solve from psi, C; the
    // instance's own descriptor (fields, diagnostics) must say the same
    virtual void set_batch_member() = 0;
    // blocked SOR tile variant (2D), see lbs_set_sor_tile
    virtual int set_sor_tile(int v) = 0;
    // all SOR rounds of a 2D solve in one launch where possible, see
    // lbs_set_sor_persistent
    virtual int set_sor_persistent(int on) = 0;
    // most polls a block waits at that form's grid barrier
    virtual int set_sor_wait_limit(long long polls) = 0;
    // step counter, total surfactant before the last rescale, rescale factor
    virtual int step_result(double *out3) = 0;
    // raw copy of the state between steps (lbs_save_state / lbs_load_state)
    virtual int save_state(void *buf, size_t *bytes) = 0;
    virtual int load_state(const void *buf, size_t bytes) = 0;
};

// parameter check shared by every entry point (message into err)
int validate_params(const lbs_params *p, char *err, size_t n);

}  // namespace lbs

struct lbs_ctx {
    lbs_params p;
    int storage;
    cudaStream_t stream;
    bool own_stream;
    void *ws;
    size_t ws_bytes;
    bool own_ws;
    lbs::Base *impl;
    char err[512];
};

namespace lbs {
// a solver for ctx->p and ctx->storage over ctx->ws on ctx->stream
Base *make_solver(lbs_ctx *ctx);
}  // namespace lbs
