// autotune.cu -- launch-shape selection for the k-sum: k-points per thread
// (KPT), threads per block and the size of a warp work item, chosen by timing
// the plan's own k-sum launches on the device.  Results are kept per context
// and, when FFE_TUNE_CACHE names a file, across processes.
//
// Key of a tuning: device name, precision, kernel variant, largest lattice N
// and log2 of the outputs per group (the amount of work that shares one
// per-k band state).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "plan.h"

namespace ffe {

static std::string tuning_key(const ffe_context* ctx, const ffe_plan* p) {
  int max_n = 2;
  double outs = 0.0;
  for (const GroupDesc& g : p->groups) {
    max_n = std::max(max_n, g.N);
    outs += g.n_out;
  }
  const int per_group = p->groups.empty() ? 0 : (int)std::lround(std::log2(std::max(1.0, outs / p->groups.size())));
  char key[256];
  snprintf(key, sizeof key, "%s|p%d|v%d|N%d|g%d", ctx->device_name.c_str(), p->prec, p->variant, max_n, per_group);
  std::string k(key);
  for (char& c : k)
    if (c == ' ') c = '_';
  return k;
}

// Defaults measured on GB300: FP32 PRODUCT 2 k-points per thread (34.7 ms
// against 46.1 ms with 4 on the N = 1024 FFLO scan; 4 would also leave room
// for only one block per SM), LIST 4 (683 ms against 736 ms with 2 on a golden
// diagram), FP64 1.
static Tuning default_tuning(int prec, int variant) {
  Tuning t;
  t.kpt = prec == FFE_FP32C ? (variant == kLayoutList ? 4 : 2) : 1;
  t.block = 256;
  t.item_target = prec == FFE_FP32C ? 8388608.0 : 262144.0;
  return t;
}

static bool valid_tuning(int prec, const Tuning& t) {
  return ksum_kpt_supported(prec, t.kpt) && (t.block == 128 || t.block == 256) && t.item_target >= 1024.0;
}

Tuning tuning_for(ffe_context* ctx, const ffe_plan* p) {
  if (p->forced) return p->tuning;
  // explicit override "kpt:block:item_target" for experiments
  if (const char* env = getenv(p->prec == FFE_FP32C ? "FFE_KSUM_TUNING_FP32" : "FFE_KSUM_TUNING_FP64")) {
    Tuning t;
    if (sscanf(env, "%d:%d:%lf", &t.kpt, &t.block, &t.item_target) == 3 && valid_tuning(p->prec, t)) return t;
  }
  auto it = ctx->tuned.find(tuning_key(ctx, p));
  if (it != ctx->tuned.end()) return it->second;
  return default_tuning(p->prec, p->variant);
}

void tuning_load(ffe_context* ctx) {
  const char* path = getenv("FFE_TUNE_CACHE");
  if (!path || !*path) return;
  ctx->tune_path = path;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[256];
  Tuning t;
  while (fscanf(f, "%255s %d %d %lf", key, &t.kpt, &t.block, &t.item_target) == 4) ctx->tuned[key] = t;
  fclose(f);
}

static void tuning_save(ffe_context* ctx) {
  if (ctx->tune_path.empty()) return;
  const std::string tmp = ctx->tune_path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : ctx->tuned)
    fprintf(f, "%s %d %d %.0f\n", kv.first.c_str(), kv.second.kpt, kv.second.block, kv.second.item_target);
  fclose(f);
  rename(tmp.c_str(), ctx->tune_path.c_str());
}

// A copy of p's inputs with a forced tuning, built without a graph.
static ffe_plan* clone_inputs(ffe_context* ctx, const ffe_plan* p, const Tuning& t) {
  ffe_plan* c = plan_new(ctx, p->kind);
  c->layout = p->layout;
  c->groups = p->groups;
  c->lines = p->lines;
  c->delta = p->delta;
  c->ht = p->ht;
  c->hlist = p->hlist;
  c->q_is_zero = p->q_is_zero;
  c->order = p->order;
  c->golden0 = p->golden0;
  c->golden_steps = p->golden_steps;
  c->n_out = p->n_out;
  c->n_q = p->n_q;
  c->n_pts = p->n_pts;
  c->forced = true;
  c->tuning = t;
  return c;
}

static std::vector<Tuning> candidates(int prec) {
  std::vector<Tuning> v;
  if (prec == FFE_FP32C) {
    for (int kpt : {2, 4, 8})
      for (double target : {2097152.0, 8388608.0, 33554432.0}) v.push_back(Tuning{kpt, 256, target});
    v.push_back(Tuning{2, 128, 8388608.0});
    v.push_back(Tuning{4, 128, 8388608.0});
  } else {
    for (int kpt : {1, 2})
      for (double target : {65536.0, 262144.0, 1048576.0}) v.push_back(Tuning{kpt, 256, target});
  }
  return v;
}

}  // namespace ffe

using namespace ffe;

extern "C" ffe_status ffe_plan_autotune(ffe_plan* p, void* stream, int32_t* kpt, int32_t* block,
                                        double* item_target) {
  if (!p) return FFE_EINVAL;
  ffe_context* ctx = p->ctx;
  (void)stream;
  double best_ms = 1e300;
  Tuning best = tuning_for(ctx, p);
  for (const Tuning& t : candidates(p->prec)) {
    ffe_plan* c = clone_inputs(ctx, p, t);
    ffe_status st = plan_configure(ctx, c);
    if (st == FFE_OK) st = plan_finish(ctx, c, false);
    double ms = 0.0;
    int32_t cnt = 0;
    // one warm-up execution, then the k-sum time of a second one
    if (st == FFE_OK) st = plan_run(ctx, c, c->stream);
    if (st == FFE_OK) st = ffe_plan_kernel_ms(c, &ms, &cnt);
    if (st == FFE_OK) st = plan_run(ctx, c, c->stream);
    if (st == FFE_OK) st = ffe_plan_kernel_ms(c, &ms, &cnt);
    if (st == FFE_OK) st = plan_check_status(ctx, c, c->stream);
    plan_free(c);
    if (st == FFE_ENOMEM) continue;  // a shape that does not fit is skipped
    if (st != FFE_OK) return st;
    if (cnt > 0 && ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  // rebuild p with the winner: build a fresh plan and swap it into p's handle
  ffe_plan* n = clone_inputs(ctx, p, best);
  ffe_status st = plan_configure(ctx, n);
  if (st == FFE_OK) st = plan_finish(ctx, n, p->exec != nullptr);
  if (st != FFE_OK) {
    plan_free(n);
    return st;
  }
  n->forced = false;
  std::swap(*p, *n);
  plan_free(n);
  ctx->tuned[tuning_key(ctx, p)] = best;
  tuning_save(ctx);
  if (kpt) *kpt = best.kpt;
  if (block) *block = best.block;
  if (item_target) *item_target = best.item_target;
  return FFE_OK;
}
