// Host/device portability macros for the numerics headers.
#pragma once
#ifdef __CUDACC__
#define STB_HD __host__ __device__ __forceinline__
#else
#define STB_HD inline
#endif
#include <cmath>
#ifndef __CUDACC__
#define __constant__
#endif
