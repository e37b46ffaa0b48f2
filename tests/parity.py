"""Decision-parity rule shared by the GPU parity tests.

A GPU sweep is compared with the FP64 oracle's sweep from the same state and
random stream.  Every gap angle must agree within ANGLE_TOL (1e-5 rad).  A
site may differ by more than that (a "flip": the two took different branches)
only when the oracle's decision at that site lay within a tolerance of its
threshold:

* the Metropolis test r < AP within PROB_TOL (1e-6) of AP;
* an angle-valued decision (the over-relaxation range test, the proposal's
  mod-2pi wrap) within ANGLE_TOL of its edge;
* the vanishing-field test (a local field shorter than FIELD_EPS leaves the
  spin unreflected) within FIELD_EPS / 2 of FIELD_EPS.

Such near-threshold decisions are counted over all checked sites and must
stay at or below NEAR_FRAC_MAX (1e-4) of them (at least one is allowed, so
that a test with fewer than 1e4 sites is not failed by a single tie).  Black
sites next to a flipped red site see a different field and are exempt from
the angle check (they are neither flips nor counted).
"""
import numpy as np

ANGLE_TOL = 1e-5      # rad
PROB_TOL = 1e-6       # Metropolis decisions within this of their threshold
NEAR_FRAC_MAX = 1e-4  # near-threshold decisions allowed per checked site
FIELD_EPS = 1e-6      # local fields shorter than this vanish (both implementations)


def near_decision(diag):
    """Mask of sites whose oracle decision lay within tolerance of a threshold
    (nan entries, i.e. sample sites, are never near)."""
    r_ap = np.abs(np.nan_to_num(diag["r_minus_ap"], nan=1.0))
    near = r_ap < PROB_TOL
    near |= np.nan_to_num(diag["or_slack"], nan=1.0) < ANGLE_TOL
    near |= np.nan_to_num(diag["wrap_slack"], nan=1.0) < ANGLE_TOL
    near |= np.abs(np.nan_to_num(diag["field"], nan=1.0) - FIELD_EPS) < 0.5 * FIELD_EPS
    return near


def _red(shape):
    yy, xx = np.mgrid[0:shape[0], 0:shape[1]]
    return ((xx + yy) & 1) == 0


def downstream_of(flip, gap):
    """Black gap sites next to a flipped red site."""
    red = _red(gap.shape)
    rf = flip & red
    t = np.zeros_like(flip)
    t[1:, :] |= rf[:-1, :]
    t[:-1, :] |= rf[1:, :]
    t[:, 1:] |= rf[:, :-1]
    t[:, :-1] |= rf[:, 1:]
    return t & ~red & (gap == 1)


class Tally:
    """Counts over one test: checked gap sites, near-threshold decisions, flips."""

    def __init__(self):
        self.sites = 0
        self.near = 0
        self.flips = 0
        self.downstream = 0

    def check_grid(self, ref, got, gap, diag, mask=False):
        """One sweep of one realisation on a whole grid.  Returns the number of
        sites whose results may differ (flips plus their downstream sites), and
        with mask=True also their mask."""
        gapm = gap == 1
        d = np.abs(np.asarray(ref, np.float64) - np.asarray(got, np.float64))
        near = near_decision(diag) & gapm
        flip = (d > ANGLE_TOL) & gapm
        down = downstream_of(flip, gap)
        flip_own = flip & ~down
        bad = flip_own & ~near
        assert not bad.any(), (
            f"{int(bad.sum())} sites differ beyond {ANGLE_TOL} rad without a decision within "
            f"tolerance of its threshold; worst {d[bad].max():.3e}, "
            f"|r - AP| there {np.abs(diag['r_minus_ap'][bad]).min():.3e}")
        self.sites += int(gapm.sum())
        self.near += int(near.sum())
        self.flips += int(flip_own.sum())
        self.downstream += int(down.sum())
        n = int(flip_own.sum() + down.sum())
        return (n, flip_own | down) if mask else n

    def check_site(self, ref, got, diag):
        """One sampled site (its neighbours taken from the GPU's own state)."""
        near = bool(near_decision({k: np.asarray(v) for k, v in diag.items()}))
        flip = abs(float(ref) - float(got)) > ANGLE_TOL
        assert not flip or near, (ref, got, diag)
        self.sites += 1
        self.near += int(near)
        self.flips += int(flip)

    def assert_budget(self):
        assert self.near <= max(1, NEAR_FRAC_MAX * self.sites), (self.near, self.sites)

    def __repr__(self):
        return (f"{self.sites} gap sites checked: {self.near} decisions within tolerance of "
                f"their threshold, {self.flips} flipped, {self.downstream} downstream")
