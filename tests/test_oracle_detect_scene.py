"""The oracle's detection step on a scene with three simultaneous emitters
(Sec. I: direct geolocation separates several emitters in one band). The
magnitude-accumulated surface thresholded at half its maximum, with a 7x7
local-maximum window, gives one detection on each emitter's node and no
other. CPU only."""
import numpy as np

import oracle
import sim


def test_crowded_scene_detections():
    s = sim.crowded()
    ref = oracle.cost_surface(*oracle.scene_args(s), acc_mode=1).reshape(121, 121)
    got = [divmod(int(k), 121) for k in oracle.detect(ref, 0.5 * ref.max(), 3)]
    assert sorted(got) == sorted(s.emitter_nodes)
    # the weak emitter is the third detection
    assert got[-1] == s.emitter_nodes[2]
