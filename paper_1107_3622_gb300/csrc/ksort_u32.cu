// Kernels and launchers of libksort for unsigned keys.
#include "ksort_launch.cuh"

template struct ksort::Launcher<unsigned>;
