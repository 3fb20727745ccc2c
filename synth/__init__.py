"""Seeded synthetic inputs for the pyramidal Lucas-Kanade hot path.

This package produces images, keypoints and camera streams only.  It holds none
of the tracking method's arithmetic (no pyramid filter, no Scharr operator, no
bilinear sampling, no Lucas-Kanade iteration, no eigenvalue test, no
forward-backward check): both the FP64 oracle and the CUDA library consume its
outputs, and neither is imported here.

Every random quantity is drawn from ``numpy.random.Generator(PCG64(seed))``.
The workloads stand in for the paper's datasets (EuRoC / NTU-VIRAL 752x480,
Botanic Garden 960x600 and 1920x1200, SubT-MRS 640x480; Sec. IV, Table III
dataset summary) with shapes, keypoint densities and motion of the same kind;
no dataset item is used or reproduced.
"""

from .texture import BlobTexture, affine_from_motion
from .keypoints import select_keypoints_topfrac, select_keypoints_nms
from .scenes import (
    Config1Pair,
    make_config1,
    HeightFieldScene,
    make_stereo_sequence,
    make_config3_pair,
    make_config3_contrast_pair,
    ContrastPair,
    StreamSpec,
    make_stream_mix,
    render_stream_frames,
    stream_rig,
)

__all__ = [
    "BlobTexture",
    "affine_from_motion",
    "select_keypoints_topfrac",
    "select_keypoints_nms",
    "Config1Pair",
    "make_config1",
    "HeightFieldScene",
    "make_stereo_sequence",
    "make_config3_pair",
    "make_config3_contrast_pair",
    "ContrastPair",
    "StreamSpec",
    "make_stream_mix",
    "render_stream_frames",
    "stream_rig",
]
