/* Error codes shared by the device runtime and the host library (values are
 * the public ones of include/gf.h). */
#ifndef GF_ERRORS_H
#define GF_ERRORS_H
#include "gf.h"
#endif
