// warmstart.h -- internal declarations of the warm-start network driver (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "internal.h"
