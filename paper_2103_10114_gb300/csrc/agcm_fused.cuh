// agcm_fused.cuh — fused stage kernel (level-streaming); see below.
#pragma once
#include "agcm_common.cuh"
