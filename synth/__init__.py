"""Seeded synthetic staircase depth frames (input generator shared by the oracle and the CUDA path)."""
from .staircase import (Camera, Frame, frame_c1, frame_c2, frame_c3, frame_c4, frame_c5,
                        frame_straight,
                        plane_frame, make_camera, straight_staircase, spiral_staircase, sense,
                        RES_C4, RES_C5, stream_pool, render_many)
from .poses import WalkFrame, tread_walk  # noqa: F401
