// Fixed-width integer types for the device code when it is compiled at run
// time (NVRTC has no C library headers).  The library's own build uses
// <cstdint> instead.
#pragma once

typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
