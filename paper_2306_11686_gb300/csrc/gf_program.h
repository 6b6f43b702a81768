/*
 * Program registry: GF_MAIN(name) registers, at load time of the object that
 * defines it, a cooperative launcher and an occupancy query for the program's
 * persistent kernel, and a launcher of its region kernel (the kernel split,
 * used when a context runs with split_regions).  Keeping the launch inside the defining translation unit
 * lets programs live in any shared object linked against the runtime.
 */
#ifndef GF_PROGRAM_H
#define GF_PROGRAM_H
#include <cuda_runtime.h>

typedef cudaError_t (*gf_launch_fn)(void **args, unsigned grid, unsigned block, void *stream);
typedef int (*gf_occ_fn)(unsigned block);

#ifdef __cplusplus
extern "C"
#endif
    __attribute__((visibility("default"))) int
    gf_program_register(const char *name, gf_launch_fn launch, gf_occ_fn occ, gf_launch_fn region);

#endif
