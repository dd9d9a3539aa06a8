// Grouped batched execution (cjt_group.cu): the stages of many transforms in one launch
// per stage and transform length class, in memory-bounded waves.
#pragma once

#include <vector>

#include "cjt_internal.cuh"

struct cjt_group_s;
typedef cjt_group_s *cjt_group_t;

// whether direction `dir` of plan p can run grouped (N >= 1, FP64 or mixed precision, no
// parameter shift, power-of-two transform lengths)
bool cjt_group_eligible(const cjt_plan_s *p, int dir);
// Lays out the items idx[] (indices into plans/dir/offsets) in waves whose workspace fits
// arena_budget bytes, allocates two arenas and the launch tables, and uploads them
// (synchronous).  *out is nullptr when idx is empty.
int cjt_group_create(cjt_group_t *out, const std::vector<int> &idx, const cjt_plan_t *plans, const int8_t *dir,
                     const int64_t *offsets, const double *in, double *outp, int64_t arena_budget);
// Enqueues every wave; forks from and joins back to `origin` (may be under stream capture).
// prof (not under capture): every launch on one stream, in order, with an event pair around
// each launch step, summed per CJT_BSTAGE_* by cjt_group_profile.
int cjt_group_issue(cjt_group_t g, cudaStream_t origin, bool prof = false);
int cjt_group_profile(cjt_group_t g, double *ms, int64_t *counts, int n);
int64_t cjt_group_kernels(cjt_group_t g);
int64_t cjt_group_arena_bytes(cjt_group_t g);
int cjt_group_waves(cjt_group_t g);
void cjt_group_destroy(cjt_group_t g);
