// agcm_adjoint.cuh — hand-written adjoint kernels of the phase decomposition.
#pragma once
#include "agcm_common.cuh"
#include "agcm_phases.cuh"
