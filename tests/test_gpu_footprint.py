"""Device memory of a chain: the Gram sums of the doubling (Eq. mu2) are one
[M/2 - 1][112] fixed-point array per chain whatever the number of CTAs, so a
chain's handle holds little beyond its two recursion buffers (2 x 7 x N
complex values), and running it allocates nothing more."""
import pytest

from paper_1303_6016_gb300 import inputs

pytestmark = pytest.mark.gpu

L = 32
BEYOND = 10e6  # bytes beyond the recursion buffers


@pytest.fixture(scope="module")
def G():
    from paper_1303_6016_gb300 import build, gfmc
    build.build()
    gfmc.load()
    return gfmc


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("M", [1024, 2048])
def test_chain_holds_little_beyond_its_vectors(G, precision, M):
    vec = 2 * 7 * L ** 3 * (16 if precision == "fp64" else 8)
    with G.Chain(L, inputs.uniform_sphere(L, 0), M=M, precision=precision, engine="grid") as ch:
        b0 = ch.device_bytes
        assert vec < b0 <= vec + BEYOND, (b0, vec)
        ch.delta_omega(5, 1.0, 1.0)
        ch.updates(2)
        assert ch.device_bytes == b0


def test_batch_growth_is_per_cta_only(G):
    """A batch on a larger team than the chain was made for (8 CTAs at L = 8)
    grows only its per-CTA words (flags, phase sums) and adds the team's tile
    plan: well under 512 bytes per CTA, nothing that scales with M."""
    tc = 16
    with G.Chain(8, inputs.uniform_sphere(8, 0), M=2048, precision="fp32_mixed") as ch:
        b0 = ch.device_bytes
        G.run_batch([ch], 1, team_ctas=[tc], trace=False)
        assert 0 < ch.device_bytes - b0 <= 512 * tc
