"""Seeded synthetic workloads shaped like the paper's experiments.

The paper's datasets (Stanford Bunny and Lounge, the robot and RGBD sequences)
are not available, so every input is generated here from a seed.  This module
holds no arithmetic of the registration method itself (no lattice, no E or M
step): it only draws point clouds, ground-truth transforms and normals, and it
imports nothing but numpy.  Both the CUDA path's tests and benchmark and the
CPU oracle's tests take their inputs from here.

All clouds are float32 arrays of shape (n, 4) (x, y, z, 0): the layout the
C-ABI takes.  Transforms are float64 (4, 4) row-major with y = T x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _pad4(p: np.ndarray) -> np.ndarray:
    out = np.zeros((p.shape[0], 4), np.float32)
    out[:, :3] = p
    return out


def random_rotation(rng: np.random.Generator, max_angle_rad: float, exact: bool = False) -> np.ndarray:
    """Rotation about a uniform axis by an angle U[0, max] (or exactly max)."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = max_angle_rad if exact else rng.uniform(0.0, max_angle_rad)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def make_T(R: np.ndarray, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def apply_T(T: np.ndarray, P: np.ndarray) -> np.ndarray:
    return (P[:, :3].astype(np.float64) @ T[:3, :3].T + T[:3, 3])


# ---------------------------------------------------------------------------
# Rigid point-to-point: bumpy sphere (2,000 + 2,000 points)
# ---------------------------------------------------------------------------

@dataclass
class RigidPair:
    X: np.ndarray            # model (M, 4)
    Y: np.ndarray            # observation (N, 4)
    T_gt: np.ndarray         # (4, 4): Y ~ T_gt X
    Yn: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def _bumpy_sphere_points(rng, n, centres, amp, width):
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    d2 = ((u[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
    r = 1.0 + amp * np.exp(-d2 / (2 * width * width)).sum(1)
    return u * r[:, None]


def sphere_bumps_pair(seed: int, n_model: int = 2000, n_obs: int = 2000, n_bumps: int = 8,
                      amp: float = 0.1, width: float = 0.2, max_angle_deg: float = 30.0,
                      max_trans: float = 0.1, noise: float = 0.005,
                      outlier_frac: float = 0.1, exact_angle: bool = False) -> RigidPair:
    """Unit sphere with Gaussian bumps; the observation is an independent sample
    of the same surface under a random rigid motion (rotation up to
    max_angle_deg about a uniform axis, exactly max_angle_deg with
    exact_angle), with isotropic noise and uniform outliers (outlier_frac *
    n_obs extra points) in its bounding box."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n_bumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    X = _bumpy_sphere_points(rng, n_model, c, amp, width)
    Ys = _bumpy_sphere_points(rng, n_obs, c, amp, width)
    R = random_rotation(rng, math.radians(max_angle_deg), exact=exact_angle)
    t = rng.uniform(-max_trans, max_trans, size=3)
    T = make_T(R, t)
    Y = Ys @ R.T + t + rng.normal(scale=noise, size=Ys.shape)
    n_out = int(round(outlier_frac * n_obs))
    if n_out:
        lo, hi = Y.min(0), Y.max(0)
        Y = np.concatenate([Y, rng.uniform(lo, hi, size=(n_out, 3))])
    Y = Y[rng.permutation(Y.shape[0])]
    return RigidPair(_pad4(X), _pad4(Y), T, None,
                     {"workload": "sphere_bumps", "seed": seed, "M": n_model, "N": Y.shape[0]})


# ---------------------------------------------------------------------------
# Rigid point-to-plane: ray-cast depth frames of a box/sphere room
# ---------------------------------------------------------------------------

@dataclass
class Scene:
    box_lo: np.ndarray       # (B, 3)
    box_hi: np.ndarray
    sph_c: np.ndarray        # (S, 3)
    sph_r: np.ndarray        # (S,)
    room: float              # half-size of the room cube


def random_scene(rng: np.random.Generator, n_objects: int = 20, room: float = 1.0,
                 keep_clear: np.ndarray | None = None, clear_radius: float = 0.35) -> Scene:
    """n_objects random axis-aligned boxes and spheres inside a 2*room cube,
    none closer than clear_radius to the point keep_clear (the camera)."""
    keep = np.zeros(3) if keep_clear is None else keep_clear
    lo, hi, sc, sr = [], [], [], []
    while len(lo) + len(sc) < n_objects:
        centre = rng.uniform(-0.8 * room, 0.8 * room, size=3)
        if rng.uniform() < 0.5:
            half = rng.uniform(0.05, 0.3, size=3)
            d = np.maximum(np.abs(keep - centre) - half, 0.0)
            if np.linalg.norm(d) < clear_radius:
                continue
            lo.append(centre - half)
            hi.append(centre + half)
        else:
            r = rng.uniform(0.05, 0.3)
            if np.linalg.norm(keep - centre) - r < clear_radius:
                continue
            sc.append(centre)
            sr.append(r)
    return Scene(np.array(lo).reshape(-1, 3), np.array(hi).reshape(-1, 3),
                 np.array(sc).reshape(-1, 3), np.array(sr), room)


def look_at_rotation(rng: np.random.Generator, forward: np.ndarray, jitter_rad: float) -> np.ndarray:
    """Camera-to-world rotation whose optical (z) axis is `forward` tilted by
    up to jitter_rad, with a random roll."""
    z = random_rotation(rng, jitter_rad) @ (forward / np.linalg.norm(forward))
    a = rng.normal(size=3)
    x = a - (a @ z) * z
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], 1)


def render_depth(scene: Scene, C: np.ndarray, W: int, H: int, fx: float, fy: float,
                 cx: float, cy: float) -> np.ndarray:
    """Analytic ray cast from the camera pose C (camera-to-world); returns the
    depth map (H, W) along the optical axis.  Every ray hits the room."""
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dc = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1).reshape(-1, 3)
    d = dc @ C[:3, :3].T
    o = C[:3, 3]
    inv = 1.0 / np.where(np.abs(d) < 1e-12, 1e-12, d)
    # The room: distance to the far wall of the cube (camera inside).
    t1 = (-scene.room - o) * inv
    t2 = (scene.room - o) * inv
    best = np.maximum(t1, t2).min(1)
    for lo, hi in zip(scene.box_lo, scene.box_hi):
        a = (lo - o) * inv
        b = (hi - o) * inv
        tn = np.minimum(a, b).max(1)
        tf = np.maximum(a, b).min(1)
        hit = (tn <= tf) & (tn > 1e-6)
        best = np.where(hit & (tn < best), tn, best)
    for c, r in zip(scene.sph_c, scene.sph_r):
        oc = o - c
        bq = d @ oc
        cq = oc @ oc - r * r
        aq = (d * d).sum(1)
        disc = bq * bq - aq * cq
        ok = disc >= 0
        tn = (-bq - np.sqrt(np.where(ok, disc, 0.0))) / aq
        hit = ok & (tn > 1e-6)
        best = np.where(hit & (tn < best), tn, best)
    return best.reshape(H, W)  # t along dc, whose z is 1: the depth


def backproject(depth: np.ndarray, fx, fy, cx, cy) -> np.ndarray:
    H, W = depth.shape
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return np.stack([(u - cx) / fx * depth, (v - cy) / fy * depth, depth], -1)


def depth_normals(P: np.ndarray) -> np.ndarray:
    """Per-pixel normals from the cross product of +-1 pixel central differences
    of the back-projected points (one-sided at the border), facing the camera."""
    Pp = np.pad(P, ((1, 1), (1, 1), (0, 0)), mode="edge")
    du = Pp[1:-1, 2:] - Pp[1:-1, :-2]
    dv = Pp[2:, 1:-1] - Pp[:-2, 1:-1]
    n = np.cross(du, dv)
    nn = np.linalg.norm(n, axis=-1, keepdims=True)
    n = n / np.where(nn > 0, nn, 1.0)
    flip = (n * P).sum(-1, keepdims=True) > 0
    return np.where(flip, -n, n)


def depth_frame_pair(seed: int, W: int = 320, H: int = 240, fx: float = 300.0, fy: float = 300.0,
                     n_objects: int = 20, max_angle_deg: float = 2.0, trans: float = 0.02,
                     depth_noise: float = 0.001, dropout: float = 0.05,
                     noise_on_model: bool = True) -> RigidPair:
    """Frame-to-frame tracking pair: X = reference frame (all W*H pixels), Y =
    the next frame after a random motion (rotation of max_angle_deg about a
    uniform axis, translation of length trans), both with N(0, depth_noise^2)
    depth noise; Y loses a random `dropout` fraction of its pixels and carries
    per-pixel normals.  Points are in each frame's camera coordinates."""
    rng = np.random.default_rng(seed)
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    # Camera 0.75 m from the room's centre, looking at the centre to within
    # 15 degrees, so that every view holds objects as well as walls.
    back = rng.normal(size=3)
    back /= np.linalg.norm(back)
    cam0 = 0.75 * back
    scene = random_scene(rng, n_objects, keep_clear=cam0)
    C0 = make_T(look_at_rotation(rng, -back, math.radians(15.0)), cam0)
    dR = random_rotation(rng, math.radians(max_angle_deg), exact=True)
    dt = rng.normal(size=3)
    dt *= trans / np.linalg.norm(dt)
    C1 = C0 @ make_T(dR, dt)                      # motion in the camera's own frame
    T_gt = np.linalg.inv(C1) @ C0                 # camera-0 coordinates -> camera-1
    d0 = render_depth(scene, C0, W, H, fx, fy, cx, cy)
    d1 = render_depth(scene, C1, W, H, fx, fy, cx, cy)
    if noise_on_model:
        d0 = d0 + rng.normal(scale=depth_noise, size=d0.shape)
    d1 = d1 + rng.normal(scale=depth_noise, size=d1.shape)
    P0 = backproject(d0, fx, fy, cx, cy)
    P1 = backproject(d1, fx, fy, cx, cy)
    N1 = depth_normals(P1)
    keep = rng.uniform(size=H * W) >= dropout
    X = _pad4(P0.reshape(-1, 3))
    Y = _pad4(P1.reshape(-1, 3)[keep])
    Yn = _pad4(N1.reshape(-1, 3)[keep])
    return RigidPair(X, Y, T_gt, Yn, {"workload": "depth_frames", "seed": seed, "W": W, "H": H,
                                      "M": X.shape[0], "N": Y.shape[0]})


def rotation_angle_deg(Ra: np.ndarray, Rb: np.ndarray) -> float:
    """Angle of Ra Rb^T in degrees (pose comparison helper)."""
    c = (np.trace(Ra[:3, :3] @ Rb[:3, :3].T) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


# ---------------------------------------------------------------------------
# Articulated: a kinematic tree of capsules
# ---------------------------------------------------------------------------

@dataclass
class KinTree:
    parent: np.ndarray       # (nb,) int32; -1 for the root (body 0)
    offset: np.ndarray       # (nb, 4, 4) joint frame of each body in its parent's frame
    joint_body: np.ndarray   # (nj,) int32, non-decreasing
    joint_axis: np.ndarray   # (nj, 3) unit axes in the frame each joint acts in
    q_min: np.ndarray        # (nj,)
    q_max: np.ndarray        # (nj,)
    radius: np.ndarray       # (nb,) capsule radius
    length: np.ndarray       # (nb,) capsule length along the body's local z

    @property
    def nb(self):
        return len(self.parent)

    @property
    def nj(self):
        return len(self.joint_body)


def _axis_rot(a, q):
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(q) * K + (1 - math.cos(q)) * (K @ K)


def pose_bodies(tree: KinTree, root_T: np.ndarray, q: np.ndarray) -> np.ndarray:
    """World transform of every body for the root pose and joint angles
    (used to place synthetic observations)."""
    T = np.zeros((tree.nb, 4, 4))
    j = 0
    for b in range(tree.nb):
        F = (root_T if b == 0 else T[tree.parent[b]]) @ tree.offset[b]
        while j < tree.nj and tree.joint_body[j] == b:
            R = np.eye(4)
            R[:3, :3] = _axis_rot(tree.joint_axis[j], q[j])
            F = F @ R
            j += 1
        T[b] = F
    return T


def random_kintree(seed: int, n_links: int = 16, n_double: int = 5, n_single: int = 10,
                   limit_deg: float = 90.0) -> KinTree:
    """A random tree of capsules (radius U[0.01, 0.03], length U[0.03, 0.1]):
    body 0 is the root; each other link hangs at the tip of a random earlier
    link, bent by up to 60 degrees; n_double links carry two orthogonal
    revolute joints, n_single links one, the rest none (6 root DOF besides)."""
    rng = np.random.default_rng(seed)
    parent = np.full(n_links, -1, np.int32)
    radius = rng.uniform(0.01, 0.03, n_links)
    length = rng.uniform(0.03, 0.1, n_links)
    offset = np.zeros((n_links, 4, 4))
    offset[0] = np.eye(4)
    for b in range(1, n_links):
        parent[b] = rng.integers(0, b)
        O = np.eye(4)
        O[:3, :3] = random_rotation(rng, math.radians(60.0))
        O[:3, 3] = [0.0, 0.0, length[parent[b]]]
        offset[b] = O
    kinds = np.array([2] * n_double + [1] * n_single + [0] * (n_links - 1 - n_double - n_single))
    rng.shuffle(kinds)
    jb, ax = [], []
    for b in range(1, n_links):
        k = kinds[b - 1]
        if k == 0:
            continue
        u = rng.normal(size=3)
        u[2] = 0.0
        u /= np.linalg.norm(u)
        jb.append(b)
        ax.append(u)
        if k == 2:
            jb.append(b)
            ax.append(np.cross([0.0, 0.0, 1.0], u))
    lim = math.radians(limit_deg)
    nj = len(jb)
    return KinTree(parent, offset, np.array(jb, np.int32), np.array(ax), np.full(nj, -lim),
                   np.full(nj, lim), radius, length)


def sample_capsules(tree: KinTree, n: int, rng: np.random.Generator):
    """n surface points of the capsules, area-proportional, in body frames:
    (points (n, 4), normals (n, 4), body ids (n,)), sorted by body."""
    area_cyl = 2 * math.pi * tree.radius * tree.length
    area_cap = 4 * math.pi * tree.radius ** 2
    area = area_cyl + area_cap
    counts = rng.multinomial(n, area / area.sum())
    P, Nn, B = [], [], []
    for b in range(tree.nb):
        c = counts[b]
        on_cyl = rng.uniform(size=c) < area_cyl[b] / area[b]
        th = rng.uniform(0, 2 * math.pi, c)
        z = rng.uniform(0, tree.length[b], c)
        u = rng.normal(size=(c, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        nrm = np.where(on_cyl[:, None], np.stack([np.cos(th), np.sin(th), np.zeros(c)], 1), u)
        cap_base = np.where((u[:, 2] >= 0)[:, None], [0.0, 0.0, 1.0], 0.0) * tree.length[b]
        pts = np.where(on_cyl[:, None], np.stack([tree.radius[b] * np.cos(th), tree.radius[b] * np.sin(th), z], 1),
                       cap_base + tree.radius[b] * u)
        P.append(pts)
        Nn.append(nrm)
        B.append(np.full(c, b, np.int32))
    return _pad4(np.concatenate(P)), _pad4(np.concatenate(Nn)), np.concatenate(B)


@dataclass
class ArticulatedPair:
    tree: KinTree
    Xref: np.ndarray         # (M, 4) model points in body frames
    body: np.ndarray         # (M,) int32
    Y: np.ndarray            # (N, 4) observation (world)
    Yn: np.ndarray           # (N, 4) observation normals
    root_gt: np.ndarray      # (4, 4)
    q_gt: np.ndarray         # (nj,)
    meta: dict = field(default_factory=dict)


def articulated_pair(seed: int, n_points: int = 30000, max_joint_deg: float = 20.0,
                     root_deg: float = 5.0, root_trans: float = 0.01, noise: float = 0.002,
                     outlier_frac: float = 0.1, tree: KinTree | None = None) -> ArticulatedPair:
    """Model: n_points capsule surface samples (body frames) at the zero pose.
    Observation: independent samples at a perturbed pose (joints U[-max, max]
    clamped to the limits; root rotated up to root_deg and moved up to
    root_trans), N(0, noise^2) noise, plus outlier_frac * n_points uniform
    outliers in the bounding box."""
    rng = np.random.default_rng(seed)
    tree = random_kintree(seed) if tree is None else tree
    Xref, _, body = sample_capsules(tree, n_points, rng)
    q_gt = np.clip(rng.uniform(-1, 1, tree.nj) * math.radians(max_joint_deg), tree.q_min, tree.q_max)
    t = rng.normal(size=3)
    t *= rng.uniform(0, root_trans) / np.linalg.norm(t)
    root_gt = make_T(random_rotation(rng, math.radians(root_deg)), t)
    Tb = pose_bodies(tree, root_gt, q_gt)
    P, Nn, B = sample_capsules(tree, n_points, rng)
    Yw = np.einsum("nij,nj->ni", Tb[B][:, :3, :3], P[:, :3]) + Tb[B][:, :3, 3]
    Nw = np.einsum("nij,nj->ni", Tb[B][:, :3, :3], Nn[:, :3])
    Yw += rng.normal(scale=noise, size=Yw.shape)
    n_out = int(round(outlier_frac * n_points))
    if n_out:
        lo, hi = Yw.min(0), Yw.max(0)
        Yw = np.concatenate([Yw, rng.uniform(lo, hi, size=(n_out, 3))])
        on = rng.normal(size=(n_out, 3))
        Nw = np.concatenate([Nw, on / np.linalg.norm(on, axis=1, keepdims=True)])
    perm = rng.permutation(Yw.shape[0])
    return ArticulatedPair(tree, Xref, body, _pad4(Yw[perm]), _pad4(Nw[perm]), root_gt, q_gt,
                           {"workload": "kintree_capsules", "seed": seed, "M": n_points,
                            "N": Yw.shape[0], "dof": 6 + tree.nj})


def posed_surface_error(pair: ArticulatedPair, root_T: np.ndarray, q: np.ndarray):
    """Mean and 99th-percentile distance between the model points posed at
    (root_T, q) and at the pair's true pose (an evaluation metric: joints that
    barely move the surface do not count against an estimate)."""
    Ta = pose_bodies(pair.tree, root_T, q)
    Tg = pose_bodies(pair.tree, pair.root_gt, pair.q_gt)
    X, B = pair.Xref[:, :3].astype(np.float64), pair.body
    Pa = np.einsum("nij,nj->ni", Ta[B][:, :3, :3], X) + Ta[B][:, :3, 3]
    Pg = np.einsum("nij,nj->ni", Tg[B][:, :3, :3], X) + Tg[B][:, :3, 3]
    d = np.linalg.norm(Pa - Pg, axis=1)
    return float(d.mean()), float(np.percentile(d, 99))


# ---------------------------------------------------------------------------
# node-graph workload: a deforming height-field surface
# ---------------------------------------------------------------------------

@dataclass
class NodeGraphPair:
    Xref: np.ndarray         # (M, 4) model points (reference surface)
    knn: np.ndarray          # (M, 4) int32: the 4 nearest nodes, nearest first
    skw: np.ndarray          # (M, 4) float32 skinning weights (rows sum to 1)
    node_pos: np.ndarray     # (K, 3) node positions (farthest-point samples of the model)
    edges: np.ndarray        # (E, 2) int32 directed node-graph edges (each node -> its 8 nearest)
    Y: np.ndarray            # (N, 4) observation: the surface resampled and deformed
    Yn: np.ndarray           # (N, 4) observation normals
    X_true: np.ndarray       # (M, 3) the model points under the true deformation
    Xn_true: np.ndarray      # (M, 3) the surface normals there (tangential motion is unobservable
                             # by point-to-plane residuals; the normal component of an error is)
    meta: dict = field(default_factory=dict)


def _height_field(rng, n_bumps):
    c = rng.uniform([-0.4, -0.3], [0.4, 0.3], size=(n_bumps, 2))
    a = rng.uniform(-0.05, 0.05, n_bumps)
    s = rng.uniform(0.03, 0.12, n_bumps)

    def surface(x, y):
        z = np.zeros_like(x)
        zx = np.zeros_like(x)
        zy = np.zeros_like(x)
        for j in range(n_bumps):
            dx, dy = x - c[j, 0], y - c[j, 1]
            g = a[j] * np.exp(-(dx * dx + dy * dy) / (2 * s[j] ** 2))
            z += g
            zx -= g * dx / s[j] ** 2
            zy -= g * dy / s[j] ** 2
        n = np.stack([-zx, -zy, np.ones_like(x)], 1)
        return np.stack([x, y, z], 1), n / np.linalg.norm(n, axis=1, keepdims=True)
    return surface


def _grid(W, H, shift):
    u = (np.arange(W) + 0.5 + shift) / W * 0.8 - 0.4
    v = (np.arange(H) + 0.5 + shift) / H * 0.6 - 0.3
    x, y = np.meshgrid(u, v)
    x, y = x.ravel(), y.ravel()
    keep = (x / 0.408) ** 2 + (y / 0.306) ** 2 <= 1.0      # ~82% of the frame
    return x[keep], y[keep]


def farthest_point_sample(P: np.ndarray, k: int, rng: np.random.Generator) -> np.ndarray:
    """Indices of k farthest-point samples of P (n, 3)."""
    idx = np.empty(k, np.int64)
    idx[0] = rng.integers(P.shape[0])
    d = np.sum((P - P[idx[0]]) ** 2, 1)
    for j in range(1, k):
        idx[j] = int(np.argmax(d))
        d = np.minimum(d, np.sum((P - P[idx[j]]) ** 2, 1))
    return idx


def nearest(P: np.ndarray, Q: np.ndarray, k: int, chunk: int = 8192):
    """The k nearest rows of Q for every row of P, nearest first: (dist, index)."""
    D = np.empty((P.shape[0], k))
    I = np.empty((P.shape[0], k), np.int64)
    q2 = np.sum(Q * Q, 1)
    for s in range(0, P.shape[0], chunk):
        p = P[s:s + chunk]
        d2 = np.maximum(np.sum(p * p, 1)[:, None] + q2[None, :] - 2.0 * p @ Q.T, 0.0)
        part = np.argpartition(d2, k - 1, axis=1)[:, :k]
        dp = np.take_along_axis(d2, part, 1)
        order = np.argsort(dp, 1)
        I[s:s + chunk] = np.take_along_axis(part, order, 1)
        D[s:s + chunk] = np.sqrt(np.take_along_axis(dp, order, 1))
    return D, I


def skinning(P: np.ndarray, node_pos: np.ndarray):
    """4 nearest nodes and weights exp(-d^2 / (2 r^2)), r = the mean distance
    from a model point to its 4 nearest nodes, normalised per point."""
    D, I = nearest(P, node_pos, 4)
    r = float(D.mean())
    w = np.exp(-D ** 2 / (2 * r * r))
    w /= w.sum(1, keepdims=True)
    return I.astype(np.int32), w.astype(np.float32), r


def nodegraph_pair(seed: int, W: int = 640, H: int = 480, n_nodes: int = 1000, n_bumps: int = 16,
                   max_disp: float = 0.03, noise: float = 0.001) -> NodeGraphPair:
    """Model: a 640x480 height field z = sum of 16 Gaussians over an
    0.8 m x 0.6 m frame, masked to an ellipse (~250k points).  Nodes:
    farthest-point samples; 4-NN skinning; each node linked to its 8 nearest
    (all others when there are fewer than 9 nodes).
    Observation: the surface resampled on the half-pixel-shifted grid and
    moved by a smooth displacement field (6 Gaussian blobs, largest
    displacement max_disp), N(0, noise^2) noise; normals carried by the
    field's Jacobian.  X_true: the model points under the same field."""
    rng = np.random.default_rng(seed)
    surface = _height_field(rng, n_bumps)
    Pm, Nm = surface(*_grid(W, H, 0.0))
    Po, No = surface(*_grid(W, H, 0.5))
    centres = rng.uniform([-0.4, -0.3, -0.05], [0.4, 0.3, 0.05], size=(6, 3))
    widths = rng.uniform(0.1, 0.25, 6)
    amps = rng.normal(size=(6, 3))

    def field_at(P):
        d = np.zeros_like(P)
        Jd = np.zeros((P.shape[0], 3, 3))
        for m in range(6):
            diff = P - centres[m]
            g = np.exp(-np.sum(diff * diff, 1) / (2 * widths[m] ** 2))
            d += g[:, None] * amps[m]
            Jd += (g[:, None, None] * amps[m][None, :, None]) * (-diff / widths[m] ** 2)[:, None, :]
        return d, Jd

    d_m, _ = field_at(Pm)
    scale = max_disp / np.linalg.norm(d_m, axis=1).max()
    amps *= scale
    d_m, J_m = field_at(Pm)
    d_o, J_o = field_at(Po)
    Yp = Po + d_o + rng.normal(scale=noise, size=Po.shape)
    F = np.eye(3)[None] + J_o
    Yn = np.einsum("nji,nj->ni", np.linalg.inv(F), No)          # (I + grad d)^-T n
    Yn /= np.linalg.norm(Yn, axis=1, keepdims=True)
    Xn = np.einsum("nji,nj->ni", np.linalg.inv(np.eye(3)[None] + J_m), Nm)
    Xn /= np.linalg.norm(Xn, axis=1, keepdims=True)
    nodes = Pm[farthest_point_sample(Pm, n_nodes, rng)]
    knn, skw, r = skinning(Pm, nodes)
    deg = min(8, n_nodes - 1)
    _, nb = nearest(nodes, nodes, deg + 1)
    edges = np.stack([np.repeat(np.arange(n_nodes), deg), nb[:, 1:].ravel()], 1).astype(np.int32)
    perm = rng.permutation(Yp.shape[0])
    return NodeGraphPair(_pad4(Pm), knn, skw, nodes, edges, _pad4(Yp[perm]), _pad4(Yn[perm]), Pm + d_m, Xn,
                         {"workload": "height_field_nodegraph", "seed": seed, "M": int(Pm.shape[0]),
                          "N": int(Yp.shape[0]), "K": n_nodes, "E": int(edges.shape[0]),
                          "skin_radius": r})


@dataclass
class FeaturePair:
    FX: np.ndarray  # (M, d) float32 model features
    FY: np.ndarray  # (N, d) float32 observation features
    Y: np.ndarray   # (N, 4) observation points
    Yn: np.ndarray  # (N, 4) observation normals
    meta: dict


def feature_frame_pair(seed: int, W: int = 320, H: int = 240, **kw) -> FeaturePair:
    """A depth-frame pair (depth_frame_pair) with the 6-d per-point feature
    [position, normal]: FX holds every model pixel's position and the normal
    of its own depth image, FY the observation's (after dropout); Y and Yn are
    the observation's points and normals."""
    p = depth_frame_pair(seed, W=W, H=H, **kw)
    Xn = depth_normals(p.X[:, :3].astype(np.float64).reshape(H, W, 3)).reshape(-1, 3)
    FX = np.concatenate([p.X[:, :3], Xn], 1).astype(np.float32)
    FY = np.concatenate([p.Y[:, :3], p.Yn[:, :3]], 1).astype(np.float32)
    return FeaturePair(np.ascontiguousarray(FX), np.ascontiguousarray(FY), p.Y, p.Yn,
                       {"workload": "depth_frames_xyz_normal", "seed": seed, "W": W, "H": H, "d": 6,
                        "M": FX.shape[0], "N": FY.shape[0]})
