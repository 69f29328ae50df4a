"""Camera matrices for rendering inputs (row-major float32 4x4, mapping
world = voxel coordinates to clip space: clip = M (x, y, z, 1)).

Input generators only, shared by the oracle tests, the GPU tests and the
benchmark; the rendering itself is not here.
"""
from __future__ import annotations

import numpy as np


def orthographic(width, height, depth=64.0):
    """World x in [0, width], y in [0, height] onto the whole viewport and
    z in [0, depth] onto depth [0, 1] (exact for dyadic sizes)."""
    m = np.zeros((4, 4), np.float32)
    m[0, 0], m[0, 3] = 2.0 / width, -1.0
    m[1, 1], m[1, 3] = 2.0 / height, -1.0
    m[2, 2], m[2, 3] = 2.0 / depth, -1.0
    m[3, 3] = 1.0
    return m


def look_at_perspective(fovy_deg, aspect, near, far, eye, target, up=(0.0, 1.0, 0.0)):
    """OpenGL-style perspective projection times a look-at view (camera
    looking down its -z axis), computed in float64, rounded to float32."""
    f = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    p = np.array([[f / aspect, 0, 0, 0], [0, f, 0, 0],
                  [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])
    z = np.asarray(eye, float) - np.asarray(target, float)
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, float), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    v = np.eye(4)
    v[:3, :3] = np.stack([x, y, z])
    v[:3, 3] = -v[:3, :3] @ np.asarray(eye, float)
    return (p @ v).astype(np.float32)


def orbit(dims, azimuth_deg, elevation_deg, distance_factor=1.6, fovy_deg=45.0, aspect=16 / 9):
    """A perspective camera on a sphere around the volume's centre, looking
    at it, far enough to see the whole volume."""
    c = np.asarray(dims, float) / 2
    r = distance_factor * float(np.linalg.norm(dims))
    az, el = np.radians(azimuth_deg), np.radians(elevation_deg)
    eye = c + r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    up = (0.0, 0.0, 1.0)
    return look_at_perspective(fovy_deg, aspect, 0.05 * r, 3.0 * r, eye, c, up)


def pinhole(eye, target, fovy_deg, aspect, up=(0.0, 0.0, 1.0)):
    """Ray-casting camera: (eye, forward, right, up) as float32 3-vectors;
    the ray of image point (u, v) in [-1, 1]^2 has direction forward +
    u * right + v * up (right and up scaled to the half field of view)."""
    f = np.asarray(target, float) - np.asarray(eye, float)
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, float))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = np.tan(np.radians(fovy_deg) / 2)
    return tuple(np.asarray(x, np.float32) for x in (eye, f, r * th * aspect, u * th))


def pinhole_orbit(dims, azimuth_deg, elevation_deg, distance_factor=1.6, fovy_deg=45.0, aspect=16 / 9):
    """A ray-casting camera on a sphere around the volume's centre."""
    c = np.asarray(dims, float) / 2
    r = distance_factor * float(np.linalg.norm(dims))
    az, el = np.radians(azimuth_deg), np.radians(elevation_deg)
    eye = c + r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    return pinhole(eye, c, fovy_deg, aspect)
