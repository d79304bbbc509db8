// hz_common.cuh -- shared device types of the step kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hz_launch.h"
#include "hz_pivot.cuh"

namespace hz {

template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };

}  // namespace hz
