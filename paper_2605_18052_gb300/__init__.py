"""GB300 epipolar pose adjustment (the hot path of FastMap's structure-from-motion stage).

The CUDA library libfastmap.so (C ABI in include/fastmap.h) holds the problem on the GPU and
runs every per-point-pair pass; this package is its Python binding plus host-side drivers.
"""
from .binding import (FM_LOSS_IRLS, FM_LOSS_L1, FM_STORE_FP16, FM_STORE_FP32, FastMapError,
                      Mlp, Options, Problem, Rotation, RotationOptions, Translation, TranslationOptions,
                      default_options, focal_vote, load_library, rotation_options, translation_options)
from .refine import Schedule, refine
from .autograd import EpipolarLoss, epipolar_loss

__all__ = ["Problem", "Mlp", "Translation", "TranslationOptions", "translation_options", "Rotation",
           "RotationOptions", "rotation_options", "Options",
           "default_options", "focal_vote", "load_library", "FastMapError", "Schedule",
           "refine", "EpipolarLoss", "epipolar_loss", "FM_STORE_FP32", "FM_STORE_FP16", "FM_LOSS_IRLS", "FM_LOSS_L1"]
