"""Host logic of the time-to-2 % measurement (plain MC against MC + denoiser)
on fakes, without a GPU: which organs count, when each loop stops, how many
decays it reports, and that the handles run one batch per checkpoint."""
import numpy as np

from paper_2111_11687_gb300 import experiment


class _Cuda:
    @staticmethod
    def synchronize():
        pass


class _Torch:
    cuda = _Cuda()

    @staticmethod
    def empty(shape, dtype=None, device=None):
        return np.zeros(shape, np.float32)

    @staticmethod
    def empty_like(a):
        return np.zeros_like(a)

    float32 = np.float32


class _Handle:
    """Organ means converging to ref as ref * (1 + c / sqrt(n)) (organ 0 ignored)."""

    def __init__(self, ref, c, opened):
        self.ref, self.c, self.n = np.asarray(ref, float), np.asarray(c, float), 0
        self.h = self
        opened.append(self)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def run(self, n, seed):
        self.n += n

    def organs(self, eps=True, sigma=True):
        assert not eps and not sigma           # organ means only
        mean = self.ref * (1.0 + self.c / np.sqrt(self.n / 1e6))
        return mean, None, None, np.full(len(self.ref), 100)

    def map_organs(self, dose):
        return dose[: len(self.ref)].astype(float)


class _Case:
    def __init__(self, ref, c):
        self.torch, self.shape, self.opened = _Torch(), (len(ref),), []
        self.ref, self.c = ref, c
        self.density = self.activity = self.labels = None
        self.nm = self

    def handle(self, **kw):
        assert kw == {"batches": 1}             # one batch per checkpoint
        return _Handle(self.ref, self.c, self.opened)

    # the nm functions the denoised loop calls
    def nm_dose_get(self, h, raw, sigma, organs):
        raw[:] = h.ref * (1.0 + h.c / np.sqrt(h.n / 1e6))


def test_organ_error_keeps_counted_organs_with_a_reference():
    means = np.array([9.0, 1.1, 2.0, 5.0, 0.7])
    ref = np.array([1.0, 1.0, 0.0, 4.0, 1.0])
    counts = np.array([50, 10, 10, 0, 10])
    err = experiment.organ_error(means, ref, counts)
    # label 0 (outside the organs), an organ without reference dose and one
    # without voxels do not count
    assert np.allclose(err, [0.1, 0.3])


def test_plain_mc_stops_at_the_first_checkpoint_within_target():
    ref = np.array([0.0, 1.0, 2.0, 3.0])
    c = np.array([0.0, 0.1, -0.19, 0.05])       # worst organ: 0.19 / sqrt(n / 1e6)
    case = _Case(ref, c)
    t, n, err = experiment.time_to_target(case, ref, 5_000_000, 10**9, 0.02, seed=1)
    # 0.19 / sqrt(n / 1e6) <= 0.02 from n = 9.025e7: the checkpoint of 9.5e7 (steps of 5e6)
    assert n == 95_000_000 and err <= 0.02 and t is not None and t >= 0
    assert len(case.opened) == 1


def test_plain_mc_gives_up_at_the_decay_limit():
    ref = np.array([0.0, 1.0])
    case = _Case(ref, np.array([0.0, 1.0]))
    t, n, err = experiment.time_to_target(case, ref, 5_000_000, 20_000_000, 0.02, seed=1)
    assert t is None and n == 20_000_000 and err > 0.02


class _Net:
    """A denoiser that shrinks the map's error by a factor."""

    def __init__(self, ref, factor):
        self.ref, self.factor = ref, factor

    def apply(self, raw, density, activity, out, roi=None):
        out[:] = self.ref + (raw - self.ref) / self.factor


def test_denoised_loop_stops_when_the_denoised_map_is_within_target():
    ref = np.array([0.0, 1.0, 2.0])
    c = np.array([0.0, 0.4, 0.1])               # raw worst error 0.4 at 1e6 decays
    case = _Case(ref, c)
    net = _Net(ref, 8.0)                        # the denoised error is 1/8 of the raw one
    t, n, err, first = experiment.time_to_target_denoised(case, net, ref, np.full(3, 100), 10_000_000,
                                                          10**9, 0.02, seed=3)
    # raw worst error at n: 0.4 / sqrt(n / 1e6); denoised / 8 <= 0.02 first at n = 1e7
    assert n == 10_000_000 and err <= 0.02 and t is not None
    e_dn, e_raw, _ = first
    assert np.isclose(e_raw.max(), 0.4 / np.sqrt(10)) and np.isclose(e_dn.max(), e_raw.max() / 8)


def test_denoised_loop_falls_back_to_more_monte_carlo():
    ref = np.array([0.0, 1.0])
    case = _Case(ref, np.array([0.0, 0.38]))
    net = _Net(ref, 2.0)
    t, n, err, first = experiment.time_to_target_denoised(case, net, ref, np.full(2, 100), 10_000_000,
                                                          10**9, 0.02, seed=3)
    # 0.19 / sqrt(n / 1e6) <= 0.02 from n = 9.025e7: the tenth checkpoint of 1e7
    assert n == 100_000_000 and err <= 0.02
