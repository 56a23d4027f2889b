// Host-side internals shared between the translation units of libskm (not exported).
#pragma once

#include "skm.h"

// Builds the sparse-row index of the resident centroid matrix now, so that skm_mem_used
// counts it (the first scoring pass that needs it builds it otherwise).
extern "C" skm_status skm_prepare_assign(skm_ctx *ctx);
