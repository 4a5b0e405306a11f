// Library-internal entry of the warm-start network used by gid_init_learned():
// one forward pass on a solver context's pitched frame planes, writing the
// predicted state (r = ln R, then T_0..T_K) into the context's pitched state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct gid_net;

int gidnet_K(const gid_net* n);

// I: 3 pitched planes (plane stride `plane` floats, row pitch `pitch`); lab:
// pitched labels; palette: K x 3 device floats; X: the state planes (same
// geometry, 3 + K + 1 planes), indirect values below tk_zero written as 0.
// Enqueued on `s`; counts kernels in *launches.
int gidnet_infer_planes(gid_net* n, int H, int W, const float* I, long plane, int pitch, const uint8_t* lab,
                        const float* palette, float tk_zero, float* X, cudaStream_t s, long long* launches,
                        std::string* err);
