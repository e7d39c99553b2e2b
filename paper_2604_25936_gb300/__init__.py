"""SAND query path on one GB300: libsand (CUDA, sm_103a) plus a thin Python binding.

SAND (arxiv 2604.25936) evaluates a tailed MLP only up to the exit layer that a
volumetric network-depth map assigns to each query point.  The C-ABI is in
include/sand.h; this package builds libsand.so in-tree and exposes it through
ctypes with PyTorch tensors for device memory and streams.
"""
from .binding import (ACT_RELU, ACT_SINE, ENC_FOURIER, ENC_NONE, FLAG_NAN_INPUT, FLAG_TIMEOUT, PRECISION,
                      RAY_HIT, RAY_MISS, RAY_NAN, RAY_STEPS, TAIL_LINEAR, TAIL_MULT, Model, SandError, SandSDF,
                      Server, lib)

__all__ = ["Model", "Server", "SandSDF", "SandError", "lib", "PRECISION", "TAIL_LINEAR", "TAIL_MULT", "ACT_SINE",
           "ACT_RELU", "ENC_NONE", "ENC_FOURIER", "FLAG_NAN_INPUT", "FLAG_TIMEOUT", "RAY_MISS", "RAY_HIT", "RAY_STEPS",
           "RAY_NAN"]
