// extern "C" entry points of include/hisa.h: argument checks and dispatch to
// the Engine; no evaluation logic lives here.
#include <new>

#include "engine.h"

struct hisa_ctx {
  hisa::Engine eng;
};

extern "C" {

hisa_status hisa_config_default(hisa_config* cfg) {
  if (!cfg) return HISA_ERR_INVALID_ARG;
  *cfg = hisa_config{};
  cfg->load_factor = 0.8f;
  cfg->ebm_k = 2.0f;
  cfg->max_iters = 1000000;
  cfg->flags = HISA_FLAG_LOG_FULL;
  cfg->device = -1;
  cfg->pull_ratio = 4.0f;
  return HISA_OK;
}

hisa_status hisa_create(const hisa_config* cfg, hisa_ctx** out) {
  if (!cfg || !out) return HISA_ERR_INVALID_ARG;
  *out = nullptr;
  hisa_ctx* c = new (std::nothrow) hisa_ctx();
  if (!c) return HISA_ERR_OOM;
  hisa_status s = c->eng.init(*cfg);
  if (s) {
    delete c;
    return s;
  }
  *out = c;
  return HISA_OK;
}

hisa_status hisa_destroy(hisa_ctx* ctx) {
  delete ctx;
  return HISA_OK;
}

hisa_status hisa_declare_relation(hisa_ctx* ctx, const char* name, uint32_t arity, int is_idb, uint32_t* rel_id) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.declare(name, arity, is_idb, rel_id);
}

hisa_status hisa_load_tuples(hisa_ctx* ctx, uint32_t rel_id, const uint32_t* const* cols, uint64_t n,
                             int cols_on_device) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.load(rel_id, cols, n, cols_on_device);
}

hisa_status hisa_add_rule(hisa_ctx* ctx, const hisa_rule* rule) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.add_rule(rule);
}

hisa_status hisa_run(hisa_ctx* ctx, hisa_run_stats* stats) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.run(stats);
}

hisa_status hisa_reset_edb(hisa_ctx* ctx) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.reset_edb();
}

hisa_status hisa_relation_size(hisa_ctx* ctx, uint32_t rel_id, uint64_t* n) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.relation_size(rel_id, n);
}

hisa_status hisa_read_relation(hisa_ctx* ctx, uint32_t rel_id, uint32_t* const* cols, uint64_t cap, uint64_t* n,
                               int cols_on_device) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.read_relation(rel_id, cols, cap, n, cols_on_device);
}

hisa_status hisa_delta_counts(hisa_ctx* ctx, uint32_t rel_id, uint64_t* out, uint32_t cap, uint32_t* n_iters) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.delta_counts(rel_id, out, cap, n_iters);
}

hisa_status hisa_load_instance(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, const uint32_t* const* cols,
                               uint64_t n, int cols_on_device) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.load_instance(rel_id, instance, cols, n, cols_on_device);
}

hisa_status hisa_instance_size(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint64_t* n) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.instance_size(rel_id, instance, n);
}

hisa_status hisa_read_instance(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint32_t* const* cols,
                               uint64_t cap, uint64_t* n, int cols_on_device) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.read_instance(rel_id, instance, cols, cap, n, cols_on_device);
}

hisa_status hisa_instance_delta_counts(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint64_t* out,
                                       uint32_t cap, uint32_t* n_iters) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.instance_delta_counts(rel_id, instance, out, cap, n_iters);
}

hisa_status hisa_serve_open(hisa_ctx* ctx, uint32_t max_instances, uint32_t max_value, uint64_t budget_bytes) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_open(max_instances, max_value, budget_bytes);
}

hisa_status hisa_serve_submit(hisa_ctx* ctx, uint32_t rel_id, const uint32_t* const* cols, uint64_t n,
                              uint64_t* ticket) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_submit(rel_id, cols, n, ticket);
}

hisa_status hisa_serve_step(hisa_ctx* ctx, uint32_t max_iterations, hisa_serve_stats* stats) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_step(max_iterations, stats);
}

hisa_status hisa_serve_poll(hisa_ctx* ctx, uint64_t ticket, int* done) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_poll(ticket, done);
}

hisa_status hisa_serve_retired(hisa_ctx* ctx, uint64_t* tickets, uint32_t cap, uint32_t* n) {
  if (!ctx || !n) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_retired(tickets, cap, n);
}

hisa_status hisa_serve_result(hisa_ctx* ctx, uint64_t ticket, uint32_t rel_id, uint32_t* const* cols, uint64_t cap,
                              uint64_t* n, uint64_t* deltas, uint32_t dcap, uint32_t* n_iters, int cols_on_device) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_result(ticket, rel_id, cols, cap, n, deltas, dcap, n_iters, cols_on_device);
}

hisa_status hisa_serve_release(hisa_ctx* ctx, uint64_t ticket) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.serve_release(ticket);
}

hisa_status hisa_kernel_stats(hisa_ctx* ctx, hisa_kernel_stat* out, uint32_t cap, uint32_t* n) {
  if (!ctx) return HISA_ERR_INVALID_ARG;
  return ctx->eng.kernel_stats(out, cap, n);
}

const char* hisa_status_string(hisa_status s) {
  switch (s) {
    case HISA_OK: return "ok";
    case HISA_ERR_INVALID_ARG: return "invalid argument";
    case HISA_ERR_ARITY: return "arity mismatch";
    case HISA_ERR_OOM: return "out of device memory";
    case HISA_ERR_NOT_CONVERGED: return "fixpoint not reached within max_iters";
    case HISA_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case HISA_ERR_CUDA: return "CUDA error";
    case HISA_ERR_UNSUPPORTED: return "unsupported rule shape";
    case HISA_ERR_STATE: return "call out of order";
    case HISA_ERR_CAPACITY: return "output buffer too small";
    case -10: return "input larger than the fixed maximum size";
    default: return "unknown status";
  }
}

const char* hisa_last_error(hisa_ctx* ctx) {
  if (!ctx) return "";
  return ctx->eng.last_error.c_str();
}

}  // extern "C"
