"""GPU versions of the generators in synth/fields.py (same values, bit for bit).

Compiled into synth/_lib/libsynth.so by ``synth.gpu.build()``.  Input
generation only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

from . import fields

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "synth_fields.cu")
LIB = os.path.join(HERE, "_lib", "libsynth.so")
_lib = None


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-cudart", "static", "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run synth.gpu.build()")
        L = ctypes.CDLL(LIB)
        P, u32, i64, u64, d = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.synth_gradient_noise.argtypes = [P, u32, u32, u32, i64, i64, i64, u64, ctypes.c_int, i64, d, d, P]
        L.synth_sphere_sdf.argtypes = [P, u32, u32, u32, i64, i64, i64, d, d, d, d, P]
        L.synth_channel_field.argtypes = [P, u32, u32, u32, i64, i64, i64, u64, u32, ctypes.c_int, i64,
                                          ctypes.c_float, ctypes.c_float, P, P]
        _lib = L
    return _lib


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def gradient_noise(nx, ny, nz, seed, octaves=6, base_period=128, gain=0.5, origin=(0, 0, 0),
                   scale=fields.NOISE_SCALE, out=None):
    import torch
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    rc = lib().synth_gradient_noise(ctypes.c_void_p(out.data_ptr()), nx, ny, nz, *origin, seed, octaves,
                                    base_period, gain, scale, _stream())
    if rc:
        raise RuntimeError(f"synth_gradient_noise failed ({rc})")
    return out


def sphere_sdf(nx, ny, nz, radius, center=None, origin=(0, 0, 0), out=None):
    import torch
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    rc = lib().synth_sphere_sdf(ctypes.c_void_p(out.data_ptr()), nx, ny, nz, *origin, *center, radius, _stream())
    if rc:
        raise RuntimeError(f"synth_sphere_sdf failed ({rc})")
    return out


def channel_field(nx, ny, nz, seed, nz_total=None, origin=(0, 0, 0), octaves=7, base_period=256, out=None):
    """GPU channel_field (window origin must be a multiple of 4 on each axis)."""
    import torch
    nz_total = nz if nz_total is None else nz_total
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    work = torch.empty(2 * nz, dtype=torch.float32, device=out.device)
    rc = lib().synth_channel_field(ctypes.c_void_p(out.data_ptr()), nx, ny, nz, *origin, seed, nz_total, octaves,
                                   base_period, float(fields.CHANNEL_GAIN), float(fields.CHANNEL_SCALE),
                                   ctypes.c_void_p(work.data_ptr()), _stream())
    if rc:
        raise RuntimeError(f"synth_channel_field failed ({rc})")
    return out


def generate(recipe, origin=(0, 0, 0), dims=None):
    """GPU counterpart of synth.recipes.generate_cpu."""
    nx, ny, nz = dims if dims is not None else recipe.dims
    if recipe.kind == "sphere":
        gx, gy, gz = recipe.dims
        return sphere_sdf(nx, ny, nz, recipe.radius, center=((gx - 1) / 2.0, (gy - 1) / 2.0, (gz - 1) / 2.0),
                          origin=origin)
    if recipe.kind == "noise":
        return gradient_noise(nx, ny, nz, recipe.seed, origin=origin)
    if recipe.kind == "channel":
        return channel_field(nx, ny, nz, recipe.seed, nz_total=recipe.dims[2], origin=origin,
                             octaves=recipe.octaves, base_period=recipe.base_period)
    raise ValueError(recipe.kind)
