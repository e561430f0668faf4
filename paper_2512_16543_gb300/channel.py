"""Seeded synthetic LEO downlink channels (system model of Section II, eqs. 1-3).

This module is the one input generator shared by the CUDA path's tests and bench and by the
FP64 oracle's tests.  It holds none of the method's arithmetic (no Gram matrix, no inverse,
no SVD, no precoder): it only produces the K x N channel matrices H(t) that both sides consume.

Model (Section II):
  * H(t) = [h_1(t), ..., h_K(t)]^T, one row per user terminal (eq. 1).
  * Rician mix h_n = sqrt(K_R/(K_R+1)) h_n^LOS + sqrt(1/(K_R+1)) h_n^NLOS (eq. 2).
  * LOS part h_n^LOS = gamma_n a(theta_n, phi_n), with the UPA manifold
    a = N^{-1/2} [exp(j kappa . r_m)]_m and kappa = 2 pi / lambda * (unit vector from the
    satellite towards the user) (eq. 3).

Readings where Section II leaves the choice open (each is listed in the design notes):
  * Fully digital array: the analog stage F_RF is the identity, so H_eff = H (eq. 4 with
    N_RF = N_t).
  * gamma_n = (h_alt / d_n(t)) exp(j psi_n): free-space loss relative to nadir and a per-user
    random phase psi_n drawn once per trajectory.
  * No range-dependent carrier phase: the user terminals compensate Doppler (Section II), so
    H(t) carries only the array-manifold change.
  * NLOS part |gamma_n(t)| g_n with g_n ~ CN(0, I_N / N) drawn once per user per trajectory,
    so the Rician K-factor holds at every step while the scatter field itself stays fixed.
  * Flat-earth local frame: the satellite starts above the disc centre at altitude h_alt,
    moves along +x at speed v; the array lies in the x-y plane, centred, element spacing
    lambda/2; users are uniform in a disc of the given radius on the ground (z = 0).

Everything is computed in float64 with torch (so the same code runs on the host for the
oracle's tests and on the device for large benches) and cast to the requested complex dtype
at the end.  All random draws come from a CPU torch.Generator seeded per call, so the
trajectory parameters do not depend on the device the channel is later evaluated on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

C_LIGHT = 299_792_458.0


@dataclass(frozen=True)
class LeoScenario:
    """Geometry and link parameters of one family of trajectories."""

    n_x: int = 8                 # UPA columns
    n_y: int = 8                 # UPA rows
    K: int = 8                   # users
    f_c: float = 20e9            # carrier frequency [Hz]
    h_alt: float = 600e3         # orbital altitude [m]
    v: float = 7.5e3             # ground-track speed [m/s]
    dt: float = 10e-3            # time between precoder updates [s]
    disc_radius: float = 50e3    # user disc radius [m]
    k_rician_db: float = 10.0    # Rician K-factor K_R [dB]
    snr_db: float = 10.0         # P_t / sigma^2 [dB]
    p_t: float = 1.0             # total transmit power P_t

    @property
    def N(self) -> int:
        return self.n_x * self.n_y

    @property
    def wavelength(self) -> float:
        return C_LIGHT / self.f_c

    @property
    def sigma2(self) -> float:
        """Noise variance so that P_t / sigma^2 equals the configured SNR."""
        return self.p_t / (10.0 ** (self.snr_db / 10.0))

    @property
    def alpha(self) -> float:
        """Classic RZF regulariser alpha = K sigma^2 / P_t (= K / SNR)."""
        return self.K * self.sigma2 / self.p_t


@dataclass
class TrajectoryParams:
    """Per-trajectory random draws (host tensors, float64 / complex128)."""

    scenario: LeoScenario
    user_xy: torch.Tensor        # [B, K, 2] ground positions [m]
    psi: torch.Tensor            # [B, K] LOS phase [rad]
    g_nlos: torch.Tensor         # [B, K, N] complex128, CN(0, I/N)
    elem_xy: torch.Tensor = field(init=False)  # [N, 2] element positions [m]

    def __post_init__(self) -> None:
        sc = self.scenario
        lam = sc.wavelength
        mx = torch.arange(sc.n_x, dtype=torch.float64) - (sc.n_x - 1) / 2.0
        my = torch.arange(sc.n_y, dtype=torch.float64) - (sc.n_y - 1) / 2.0
        gy, gx = torch.meshgrid(my, mx, indexing="ij")   # element m = m_y * n_x + m_x
        self.elem_xy = torch.stack([gx.reshape(-1), gy.reshape(-1)], dim=-1) * (lam / 2.0)

    @property
    def batch(self) -> int:
        return self.user_xy.shape[0]


def draw_trajectories(scenario: LeoScenario, batch: int, seed: int,
                      radius: torch.Tensor | None = None) -> TrajectoryParams:
    """Draw user positions, LOS phases and NLOS fields for `batch` independent trajectories.

    radius: optional per-trajectory disc radius [batch] in metres (default: the scenario's).
    """
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    K, N = scenario.K, scenario.N
    u = torch.rand(batch, K, generator=g, dtype=torch.float64)
    ang = torch.rand(batch, K, generator=g, dtype=torch.float64) * (2.0 * math.pi)
    r_disc = (scenario.disc_radius if radius is None
              else radius.to(torch.float64).reshape(batch, 1))
    rad = r_disc * torch.sqrt(u)
    user_xy = torch.stack([rad * torch.cos(ang), rad * torch.sin(ang)], dim=-1)
    psi = torch.rand(batch, K, generator=g, dtype=torch.float64) * (2.0 * math.pi)
    re = torch.randn(batch, K, N, generator=g, dtype=torch.float64)
    im = torch.randn(batch, K, N, generator=g, dtype=torch.float64)
    g_nlos = torch.complex(re, im) * math.sqrt(0.5 / N)
    return TrajectoryParams(scenario, user_xy, psi, g_nlos)


def channel_at(params: TrajectoryParams, t: int, *, device="cpu",
               dtype: torch.dtype = torch.complex128,
               index: torch.Tensor | None = None) -> torch.Tensor:
    """H(t) for every trajectory (or the subset `index`): tensor [B, K, N] of `dtype`.

    Time t is the precoder-update index; the satellite sits at x = v * t * dt.
    """
    sc = params.scenario
    user_xy, psi, g_nlos = params.user_xy, params.psi, params.g_nlos
    if index is not None:
        user_xy, psi, g_nlos = user_xy[index], psi[index], g_nlos[index]
    user_xy = user_xy.to(device)
    psi = psi.to(device)
    g_nlos = g_nlos.to(device)
    elem_xy = params.elem_xy.to(device)

    x_sat = sc.v * sc.dt * float(t)
    dx = user_xy[..., 0] - x_sat                       # [B, K]
    dy = user_xy[..., 1]
    dz = torch.full_like(dx, -sc.h_alt)
    dist = torch.sqrt(dx * dx + dy * dy + dz * dz)
    ux, uy = dx / dist, dy / dist                      # direction cosines of departure
    k0 = 2.0 * math.pi / sc.wavelength
    phase = k0 * (ux[..., None] * elem_xy[:, 0] + uy[..., None] * elem_xy[:, 1])  # [B,K,N]
    a = torch.polar(torch.full_like(phase, 1.0 / math.sqrt(sc.N)), phase)
    gain = sc.h_alt / dist                             # |gamma_n|
    gamma = torch.polar(gain, psi)                     # gamma_n
    kr = 10.0 ** (sc.k_rician_db / 10.0)
    h_los = gamma[..., None] * a
    h_nlos = gain[..., None].to(torch.complex128) * g_nlos
    H = math.sqrt(kr / (kr + 1.0)) * h_los + math.sqrt(1.0 / (kr + 1.0)) * h_nlos
    return H.to(dtype).contiguous()


def steering_at(params: TrajectoryParams, t: int, *, device="cpu") -> torch.Tensor:
    """The array-manifold vectors a(theta_n(t), phi_n(t)) of eq. 3 (no gain, no NLOS part):
    [B, K, N] complex128.  This is the geometric channel the satellite knows from positions
    (Section II), the input of the digital precoder in the hybrid case."""
    sc = params.scenario
    user_xy = params.user_xy.to(device)
    elem_xy = params.elem_xy.to(device)
    x_sat = sc.v * sc.dt * float(t)
    dx = user_xy[..., 0] - x_sat
    dy = user_xy[..., 1]
    dist = torch.sqrt(dx * dx + dy * dy + sc.h_alt * sc.h_alt)
    k0 = 2.0 * math.pi / sc.wavelength
    phase = k0 * ((dx / dist)[..., None] * elem_xy[:, 0] + (dy / dist)[..., None] * elem_xy[:, 1])
    return torch.polar(torch.full_like(phase, 1.0 / math.sqrt(sc.N)), phase)


def dft_codebook(scenario: LeoScenario, *, device="cpu") -> torch.Tensor:
    """Orthonormal 2-D DFT codebook of the UPA (Section II eq. 4): column (p, q) steers to the
    direction cosines (-1 + 2p / n_x, -1 + 2q / n_y) on the lambda/2 grid; [N, N] complex128,
    column index p * n_y + q."""
    nx, ny = scenario.n_x, scenario.n_y
    mx = torch.arange(nx, dtype=torch.float64, device=device) - (nx - 1) / 2.0
    my = torch.arange(ny, dtype=torch.float64, device=device) - (ny - 1) / 2.0
    gy, gx = torch.meshgrid(my, mx, indexing="ij")          # element m = m_y * n_x + m_x
    ux = -1.0 + 2.0 * torch.arange(nx, dtype=torch.float64, device=device) / nx
    uy = -1.0 + 2.0 * torch.arange(ny, dtype=torch.float64, device=device) / ny
    bx, by = torch.meshgrid(ux, uy, indexing="ij")           # beam (p, q)
    phase = math.pi * (gx.reshape(-1, 1) * bx.reshape(1, -1) +
                       gy.reshape(-1, 1) * by.reshape(1, -1))
    return torch.polar(torch.full_like(phase, 1.0 / math.sqrt(nx * ny)), phase)


def best_power_beams(steer: torch.Tensor, codebook: torch.Tensor) -> torch.Tensor:
    """Per user the codebook column with the largest |a_n^H f|^2 (best-power selection of
    Section II): steer [B, K, N], codebook [N, M] -> beam indices [B, K]."""
    return torch.argmax((steer.conj() @ codebook).abs(), dim=-1)


def hybrid_channels(params: TrajectoryParams, t: int, codebook: torch.Tensor, *, device="cpu",
                    dtype: torch.dtype = torch.complex128):
    """Hybrid beamforming at snapshot t with N_RF = K (one beam per user, best power):
    returns (H_eff, H_true_eff, F_RF).  H_eff = A F_RF [B, K, K] is the geometric effective
    channel the digital precoder is computed from (eq. 4, A = the steering vectors), in `dtype`;
    H_true_eff = H F_RF [B, K, K] (complex128) is the Rician channel of eqs. 1-3 seen through the
    same beams (for the sum-rate of eq. 15); F_RF [B, N, K] complex128."""
    cb = codebook.to(device)
    A = steering_at(params, t, device=device)
    beams = best_power_beams(A.to(torch.complex64), cb.to(torch.complex64))
    F = cb[:, beams].permute(1, 0, 2)                        # [B, N, K]
    H = channel_at(params, t, device=device, dtype=torch.complex128)
    return (A @ F).to(dtype).contiguous(), (H @ F).contiguous(), F


def trajectory(params: TrajectoryParams, steps: int, *, t0: int = 0, device="cpu",
               dtype: torch.dtype = torch.complex128) -> torch.Tensor:
    """Stack H(t0), ..., H(t0+steps-1): tensor [steps, B, K, N]."""
    return torch.stack([channel_at(params, t0 + s, device=device, dtype=dtype)
                        for s in range(steps)])


# Named workloads (sizes of the five standard configurations).  Only the scenario and batch
# are fixed here; precision and rank-rule settings live with the callers.
def scenario_single_small() -> LeoScenario:
    """8x8 UPA (N=64) at 20 GHz, K=8 users in a 50 km disc, SNR 10 dB."""
    return LeoScenario(n_x=8, n_y=8, K=8, disc_radius=50e3, snr_db=10.0)


def scenario_batched_256x32() -> LeoScenario:
    """16x16 UPA (N=256) at 20 GHz, K=32 users in a 50 km disc, SNR 10 dB."""
    return LeoScenario(n_x=16, n_y=16, K=32, disc_radius=50e3, snr_db=10.0)


def scenario_large_4096x512() -> LeoScenario:
    """64x64 UPA (N=4096), K=512 users in a 300 km disc, SNR 10 dB."""
    return LeoScenario(n_x=64, n_y=64, K=512, disc_radius=300e3, snr_db=10.0)


@dataclass
class UnevenClass:
    """The instances of one (N, K) class of an uneven population."""

    scenario: LeoScenario        # array and K; its disc radius and SNR are not used
    index: torch.Tensor          # [B_c] positions in the mixed population
    radius: torch.Tensor         # [B_c] user-disc radius [m]
    snr_db: torch.Tensor         # [B_c] P_t / sigma^2 [dB]
    params: TrajectoryParams

    @property
    def batch(self) -> int:
        return int(self.index.numel())

    @property
    def sigma2(self) -> list[float]:
        return [self.scenario.p_t / 10.0 ** (float(x) / 10.0) for x in self.snr_db]

    @property
    def alpha(self) -> list[float]:
        """Per-instance RZF regulariser K sigma^2 / P_t."""
        return [self.scenario.K * s / self.scenario.p_t for s in self.sigma2]


UNEVEN_ARRAYS = {256: (16, 16), 512: (32, 16), 1024: (32, 32)}


def uneven_population(count: int, seed: int, *, n_choices=(256, 512, 1024),
                      k_choices=(16, 32, 64, 128), radius_km=(20.0, 200.0),
                      snr_db=(0.0, 20.0)) -> list[UnevenClass]:
    """`count` instances, each with (N, K) drawn uniformly from the choices, its own user-disc
    radius ~ U(radius_km) and SNR ~ U(snr_db); grouped by (N, K) class (classes in a fixed
    order, instances in population order)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    ni = torch.randint(len(n_choices), (count,), generator=g)
    ki = torch.randint(len(k_choices), (count,), generator=g)
    rad = (radius_km[0] + (radius_km[1] - radius_km[0]) *
           torch.rand(count, generator=g, dtype=torch.float64)) * 1e3
    snr = snr_db[0] + (snr_db[1] - snr_db[0]) * torch.rand(count, generator=g,
                                                           dtype=torch.float64)
    out = []
    for a, N in enumerate(n_choices):
        for b, K in enumerate(k_choices):
            idx = torch.nonzero((ni == a) & (ki == b)).flatten()
            if idx.numel() == 0:
                continue
            nx, ny = UNEVEN_ARRAYS[N]
            sc = LeoScenario(n_x=nx, n_y=ny, K=K)
            params = draw_trajectories(sc, int(idx.numel()), seed=seed * 1000 + 10 * a + b,
                                       radius=rad[idx])
            out.append(UnevenClass(sc, idx, rad[idx], snr[idx], params))
    return out


def scenario_paper_hybrid(K: int = 16, snr_db: float = 10.0) -> LeoScenario:
    """Section VI / Table III: 18 GHz, 600 km, 16x16 UPA at lambda/2, N_RF = K <= 16 beams,
    K_R = 10 dB, updates every 50 ms (users: draw_beam_users, one per beam cell).  The paper
    gives no noise bandwidth, so P_t / sigma^2 is a parameter: 10 dB as in the other workloads;
    about 30 dB is the order of Table III's link budget (P_t = 20 dBW, UT gain 39.7 dBi,
    173 dB free-space loss, a few hundred MHz of noise) with the array gain inside
    |a^H f|^2 <= 1."""
    return LeoScenario(n_x=16, n_y=16, K=K, f_c=18e9, dt=50e-3, disc_radius=250e3,
                       snr_db=snr_db)


def draw_beam_users(scenario: LeoScenario, batch: int, seed: int,
                    beams: tuple = (6, 7, 8, 9)) -> TrajectoryParams:
    """Users for the hybrid case, one per DFT beam (Table III: one active user per beam): user
    k of each trajectory is uniform inside the cell of beam (p_k, q_k), p, q over `beams` (the
    cells of direction cosines (-1 + 2p / n_x +- 1 / n_x, ...) seen from the satellite at
    t = 0), mapped to the ground; K must equal len(beams)^2.  LOS phases and NLOS fields are
    drawn as in draw_trajectories."""
    K, nx, ny = scenario.K, scenario.n_x, scenario.n_y
    cells = [(p, q) for p in beams for q in beams]
    if len(cells) != K:
        raise ValueError("K must equal the number of beam cells")
    base = draw_trajectories(scenario, batch, seed)
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) + 7)
    jit = torch.rand(batch, K, 2, generator=g, dtype=torch.float64) * 2.0 - 1.0
    cu = torch.tensor([[-1.0 + 2.0 * p / nx, -1.0 + 2.0 * q / ny] for p, q in cells],
                      dtype=torch.float64)
    half = torch.tensor([1.0 / nx, 1.0 / ny], dtype=torch.float64)
    u = cu + jit * half                                       # direction cosines [B, K, 2]
    uz = torch.sqrt(1.0 - (u * u).sum(-1, keepdim=True))
    user_xy = scenario.h_alt * u / uz                         # ground point seen at (ux, uy)
    return TrajectoryParams(scenario, user_xy, base.psi, base.g_nlos)
