"""Host-side pieces of the learned encoder aid that need no GPU: the PSNR
of Eq. 4-5 used in its reports, against the oracle's."""
import numpy as np

import lf_synth
import oracle
from paper_1805_06019_gb300 import learned


def test_psnr_matches_the_oracle():
    lf = lf_synth.make_lightfield(3, 3, 20, 12, [0.0, 1.0], 1.0, preset_id=700)
    rng = np.random.default_rng(1)
    dec = np.clip(lf.astype(int) + rng.integers(-3, 4, lf.shape), 0, 255).astype(np.uint8)
    assert abs(learned.psnr_ycocg(lf, dec) - oracle.psnr_ycocg(lf, dec)) < 1e-9
    assert learned.psnr_ycocg(lf, lf) == oracle.psnr_ycocg(lf, lf) == 99.0
