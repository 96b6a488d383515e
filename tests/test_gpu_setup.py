"""Set-up validation through the C ABI (GPU: a context needs a device).

The geometry checks run when the context is set up (first step or read): a
fluid node may lie on at most one non-periodic box face, and that face must
carry a velocity or pressure condition; the first offending node in node
order (x fastest) is the one reported.  Tag values other than 0 and 1 are
refused when the geometry is set."""
import numpy as np
import pytest

from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300.binding import ERR_ARG, FACE_PRESSURE, FACE_VELOCITY, IBLError, Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _duct():
    return G.straight_duct(16, 10, 10, 6.0, u_max=0.02)


def _duct_solver(tag):
    g = _duct()
    s = Solver(g.nx, g.ny, g.nz, 0.8)
    s.set_geometry(tag if tag is not None else g.tag, g.links)
    for face, spec in enumerate(g.faces):
        if spec.kind == FACE_VELOCITY:
            s.set_inlet_velocity(face, spec.velocity)
        elif spec.kind == FACE_PRESSURE:
            s.set_outlet_pressure(face, spec.rho)
    return g, s


def _node(g, x, y, z):
    return x + g.nx * (y + g.ny * z)


def test_tag_values_other_than_0_and_1_are_refused():
    g = _duct()
    s = Solver(g.nx, g.ny, g.nz, 0.8)
    for at in (0, 7, 8, g.n_nodes - 1):          # inside a word and in the tail
        tag = np.array(g.tag, np.uint8)
        tag[at] = 2
        with pytest.raises(IBLError) as e:
            s.set_geometry(tag, g.links)
        assert e.value.status == ERR_ARG and "cell_tag" in str(e.value)
    s.set_geometry(g.tag, g.links)
    s.close()


def test_first_fluid_node_on_a_face_without_condition_is_reported():
    g = _duct()
    tag = np.array(g.tag, np.uint8)
    lo, hi = _node(g, 5, 0, 5), _node(g, 9, 0, 7)   # on face y- (face 2), which has no condition
    tag[hi] = 0
    tag[lo] = 0
    _, s = _duct_solver(tag)
    with pytest.raises(IBLError) as e:
        s.step(1)
    msg = str(e.value)
    assert e.value.status == ERR_ARG and f"fluid node {lo} lies on face 2" in msg, msg
    s.close()


def test_fluid_node_on_a_box_edge_is_reported():
    g = _duct()
    tag = np.array(g.tag, np.uint8)
    n = _node(g, 0, 0, 4)                           # on faces x- and y-
    tag[n] = 0
    tag[_node(g, 7, 9, 9)] = 0                      # a later node on two faces too
    _, s = _duct_solver(tag)
    with pytest.raises(IBLError) as e:
        s.step(1)
    msg = str(e.value)
    assert e.value.status == ERR_ARG and f"fluid node {n} lies on an edge" in msg, msg
    s.close()


def test_valid_duct_sets_up():
    _, s = _duct_solver(None)
    done, _ = s.step(2)
    assert done == 2
    s.close()


def _capsule_in_duct(tris_edit):
    from paper_2207_06043_gb300 import meshes as Ms
    g = G.straight_duct(24, 16, 16, 12.0, u_max=0.02)
    V, T = Ms.sphere_mesh(162, 6.0, (8.0, g.info["yc"], g.info["zc"]), Ms.SplitMix64(2))
    s = Solver.from_geometry(g, 0.8, u_max=0.02)
    return s, V, tris_edit(np.array(T, np.int32))


def test_capsule_index_errors_are_reported_when_added():
    def bad(T):
        T[3, 1] = T[3, 0]            # a triangle with a repeated vertex
        return T
    s, V, T = _capsule_in_duct(bad)
    with pytest.raises(IBLError) as e:
        s.add_capsule(V, T)
    assert e.value.status == ERR_ARG and "triangle 3 has an invalid vertex index" in str(e.value)
    T[3, 1] = len(V)                 # out of range
    with pytest.raises(IBLError):
        s.add_capsule(V, T)
    s.close()


@pytest.mark.parametrize("edit,words", [
    (lambda T: T[1:], "not closed"),                                     # a triangle missing
    (lambda T: np.concatenate([T[:1, ::-1], T[1:]]), "same direction"),  # one triangle flipped
])
def test_open_or_misoriented_capsule_is_reported_at_set_up(edit, words):
    s, V, T = _capsule_in_duct(edit)
    s.add_capsule(V, T)              # accepted here
    s.add_capsule(V + 0.0, T)        # a second one, so the message must name the first
    with pytest.raises(IBLError) as e:
        s.step(1)
    msg = str(e.value)
    assert e.value.status == ERR_ARG and "capsule 0 mesh" in msg and words in msg, msg
    s.close()
