"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds geometry and input generation only (rooms, patches, candidate points,
lamp source layouts, dwell vectors); none of the irradiance arithmetic.
"""
from .scenes import (Lamp, Scene, dwell_vectors, large_floor, line_lamp,  # noqa: F401
                     point_lamp, tiny_room, ward_room)
