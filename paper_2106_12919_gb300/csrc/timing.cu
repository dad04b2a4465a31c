// Per-stage device timing with CUDA events on the context stream, and launch counts.
#include "pic_internal.cuh"

namespace {
const char* kStageNames[STAGE_COUNT] = {"push", "fft", "update", "bin", "other"};
constexpr int kPool = 1 << 14;  // event pairs
}  // namespace

StageScope::StageScope(pic_ctx* c, int stage, int launches) : ctx(c), pair(-1) {
  ctx->timers.launches[stage] += launches;
  Timers& t = ctx->timers;
  if (t.on && t.used < t.pool_size) {
    pair = t.used++;
    t.stage[pair] = stage;
    cudaEventRecord(t.pool[2 * pair], ctx->stream);
  }
}

StageScope::~StageScope() {
  if (pair >= 0) cudaEventRecord(ctx->timers.pool[2 * pair + 1], ctx->stream);
}

void timers_free(pic_ctx* ctx) {
  Timers& t = ctx->timers;
  if (t.pool) {
    for (int i = 0; i < 2 * t.pool_size; ++i) cudaEventDestroy(t.pool[i]);
    delete[] t.pool;
    delete[] t.stage;
  }
  t.pool = nullptr;
  t.stage = nullptr;
  t.pool_size = 0;
}

extern "C" pic_status pic_timing(pic_ctx* ctx, int enable) {
  if (!ctx) return PIC_ERR_ARG;
  Timers& t = ctx->timers;
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < STAGE_COUNT; ++s) t.launches[s] = 0;
  t.used = 0;
  t.on = enable ? 1 : 0;
  if (enable && !t.pool) {
    t.pool = new cudaEvent_t[2 * kPool];
    t.stage = new int[kPool];
    for (int i = 0; i < 2 * kPool; ++i) PIC_CUDA_TRY(ctx, cudaEventCreate(&t.pool[i]));
    t.pool_size = kPool;
  }
  return PIC_OK;
}

extern "C" pic_status pic_timing_read(pic_ctx* ctx, const char* stage, double* ms, int64_t* launches) {
  if (!ctx) return PIC_ERR_ARG;
  if (!stage || !ms || !launches) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  Timers& t = ctx->timers;
  int which = -1;
  for (int s = 0; s < STAGE_COUNT; ++s)
    if (strcmp(stage, kStageNames[s]) == 0) which = s;
  if (which < 0 && strcmp(stage, "all") != 0) return pic_set_error(ctx, PIC_ERR_ARG, "unknown stage '%s'", stage);
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  double total = 0.0;
  int64_t n = 0;
  for (int s = 0; s < STAGE_COUNT; ++s)
    if (which < 0 || s == which) n += t.launches[s];
  for (int i = 0; i < t.used; ++i) {
    if (which >= 0 && t.stage[i] != which) continue;
    float e = 0.0f;
    PIC_CUDA_TRY(ctx, cudaEventElapsedTime(&e, t.pool[2 * i], t.pool[2 * i + 1]));
    total += e;
  }
  *ms = total;
  *launches = n;
  return PIC_OK;
}
