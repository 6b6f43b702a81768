/*
 * Library-internal hooks between the host runtime (runtime.cu) and the
 * executors that launch their own kernels (synthetic loops).  Not exported.
 */
#ifndef GF_INTERNAL_H
#define GF_INTERNAL_H
#include "gf.h"
#include "gf_layout.h"

/* borrow a free program instance: state initialised, ring segment served */
gf_state *gf_inst_acquire(gf_ctx *c, void *stream, uint32_t nblocks, int *idx);
/* give it back (the caller's stream must be drained) */
void gf_inst_release(gf_ctx *c, int idx);
/* device scratch of the instance (its reduction-partials array, >= 16 KiB) */
void *gf_inst_scratch(gf_ctx *c, int idx);
int gf_ctx_server_threads(gf_ctx *c);
/* the instance's heap arena (device) and its size */
void gf_inst_heap(gf_ctx *c, int idx, void **base, uint64_t *bytes);
#endif
