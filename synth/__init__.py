"""Seeded synthetic inputs: PF-element events and model weight blobs.

This module is shared by the FP64 oracle, the tests and the benchmark.  It holds
no arithmetic of the MLPF method itself: only a counter-based random generator,
the event generator, the seeded weight initialiser and the weight-blob writer.

Random numbers come from one counter-based generator, the SplitMix64 output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied as a hash of a key tuple, so that every value is a pure
function of (seed, stream, index...) and any element can be regenerated alone.

Events (Sec. 5.2 features; size statistics mimic the Run-3 pileup samples of
Sec. 4, about 5000 elements per event per Sec. 5.3):
  x[:, 0:8]   one-hot element type: track, ECAL, HCAL, HF-EM, HF-HAD, GSF track,
              brem, supercluster (drawn with probabilities 40/25/20/3/3/3/3/3 %)
  x[:, 8]     log pT  ~ N(0, 1)   (log GeV)
  x[:, 9]     log E   ~ N(0, 1)   (log GeV)
  x[:, 10]    eta: tracks, GSF tracks, brem U[-2.5, 2.5]; HF U[-5, 5];
              ECAL, HCAL, supercluster U[-3, 3]
  x[:, 11:13] sin phi, cos phi with phi ~ U[-pi, pi]
  x[:, 13:30] 17 track-only features ~ N(0,1), zero for calorimeter types
  x[:, 30:42] 12 cluster-only features ~ N(0,1), zero for track types
"""
from __future__ import annotations

import dataclasses
import math
import struct

import numpy as np

IN_DIM = 42
N_TYPES = 8
N_CLS = 6
N_REG = 5
TYPE_NAMES = ("track", "ecal", "hcal", "hf_em", "hf_had", "gsf", "brem", "sc")
TYPE_PROBS = (0.40, 0.25, 0.20, 0.03, 0.03, 0.03, 0.03, 0.03)
TRACK_TYPES = (0, 5, 6)
CLUSTER_TYPES = (1, 2, 3, 4, 7)
CLASS_NAMES = ("none", "ch_had", "n_had", "photon", "electron", "muon")

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (first key word after the seed)
STREAM_EVENT_SIZE = 1
STREAM_ELEMENT = 2
STREAM_WEIGHT = 3


def splitmix64(z):
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def hash_key(*words):
    """Hash a tuple of integer (array) words into one uint64 per element."""
    h = splitmix64(np.uint64(0))
    for w in words:
        h = splitmix64(h ^ np.asarray(w, dtype=np.uint64))
    return h


def uniform(*words):
    """U[0,1) double from the top 53 bits of hash_key(words)."""
    h = hash_key(*words)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(*words):
    """N(0,1) by Box-Muller from two sub-keys of words (sub-key 0 and 1)."""
    u1 = uniform(*words, 0)
    u2 = uniform(*words, 1)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# event sizes
# --------------------------------------------------------------------------

def sizes_uniform(seed: int, n_events: int, lo: int = 1000, hi: int = 6000):
    """N ~ U{lo..hi} per event (pileup-like size mix)."""
    e = np.arange(n_events, dtype=np.uint64)
    u = uniform(seed, STREAM_EVENT_SIZE, e)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def sizes_lognormal(seed: int, n_events: int, median: float = 2500.0,
                    sigma: float = 0.5, lo: int = 100, hi: int = 12000):
    """N ~ LogNormal(ln median, sigma), rounded and clipped to [lo, hi]."""
    e = np.arange(n_events, dtype=np.uint64)
    z = normal(seed, STREAM_EVENT_SIZE, e)
    n = np.rint(np.exp(math.log(median) + sigma * z))
    return np.clip(n, lo, hi).astype(np.int64)


# --------------------------------------------------------------------------
# events
# --------------------------------------------------------------------------

def gen_events(seed: int, sizes, first_event: int = 0):
    """Packed events: x [T, 42] float32 and cu_seqlens [n+1] int32.

    Element i of event e depends only on (seed, first_event + e, i), so a large
    set can be generated in independent chunks.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    cu = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=cu[1:])
    total = int(cu[-1])
    ev = np.repeat(np.arange(len(sizes), dtype=np.uint64) + np.uint64(first_event), sizes)
    idx = (np.arange(total, dtype=np.int64) - np.repeat(cu[:-1], sizes)).astype(np.uint64)
    x = np.zeros((total, IN_DIM), dtype=np.float32)
    if total == 0:
        return x, cu.astype(np.int32)

    def U(slot):
        return uniform(seed, STREAM_ELEMENT, ev, idx, slot)

    def Nrm(slot):
        return normal(seed, STREAM_ELEMENT, ev, idx, slot)

    u_type = U(0)
    edges = np.cumsum(TYPE_PROBS)
    edges[-1] = 1.0 + 1e-12
    typ = np.searchsorted(edges, u_type, side="right")
    x[np.arange(total), typ] = 1.0
    x[:, 8] = Nrm(1)
    x[:, 9] = Nrm(2)
    ueta = U(3) * 2.0 - 1.0
    eta_half = np.where(np.isin(typ, (3, 4)), 5.0,
                        np.where(np.isin(typ, (1, 2, 7)), 3.0, 2.5))
    x[:, 10] = ueta * eta_half
    phi = (U(4) * 2.0 - 1.0) * math.pi
    x[:, 11] = np.sin(phi)
    x[:, 12] = np.cos(phi)
    is_trk = np.isin(typ, TRACK_TYPES)
    for k in range(17):
        x[:, 13 + k] = np.where(is_trk, Nrm(10 + k), 0.0)
    for k in range(12):
        x[:, 30 + k] = np.where(~is_trk, Nrm(40 + k), 0.0)
    return x, cu.astype(np.int32)


# --------------------------------------------------------------------------
# model configuration and weights
# --------------------------------------------------------------------------

ACT_GELU = 0
ACT_RELU = 1


@dataclasses.dataclass(frozen=True)
class ModelConfig:
    d: int = 64
    heads: int = 4
    ffn: int = 256
    l_pid: int = 1
    l_reg: int = 1
    act: int = ACT_GELU
    in_dim: int = IN_DIM
    n_cls: int = N_CLS
    n_reg: int = N_REG
    # ARCH_SEQ: one shared embedding, the regression stack reads concat(x, h_pid),
    # one 6-class head.  ARCH_PAPER (Sec. 5.3 as printed): track and cluster
    # embeddings, two parallel stacks on the same embedding, binary + 5-class PID
    # heads (class-score columns: [binary logit, 5 PID logits]).
    arch: int = 0

    @property
    def dh(self) -> int:
        return self.d // self.heads


ARCH_SEQ, ARCH_PAPER = 0, 1

# The architecture of the 1-event / 64-event / 512-event workloads.
SMALL = ModelConfig(d=64, heads=4, ffn=256, l_pid=1, l_reg=1)
# The full-size architecture (d=256, 8 heads of 32, FFN 1024, 3+3 layers).
FULL = ModelConfig(d=256, heads=8, ffn=1024, l_pid=3, l_reg=3)

# The architecture as Sec. 5.3 prints it: d=256, 16 heads of 16, ReLU, 3+3 blocks
# (FFN width unstated: 4 d), per-type embedding, parallel encoders, binary + PID heads.
PAPER = ModelConfig(d=256, heads=16, ffn=1024, l_pid=3, l_reg=3, act=ACT_RELU, arch=ARCH_PAPER)

# Output width of each regression head, in output-column order.
REG_HEADS = (("pt", 1), ("eta", 1), ("phi", 2), ("e", 1))


def tensor_specs(cfg: ModelConfig):
    """Ordered (name, shape, kind) of every parameter tensor.

    kind: 'w' Xavier-initialised matrix [out, in]; 'b' bias; 'g' LN gain;
    'beta' LN shift.  The order fixes the random stream index of each tensor.
    """
    d, f = cfg.d, cfg.ffn
    paper = cfg.arch == ARCH_PAPER

    def mlp(prefix, n_in, n_out):
        return [(prefix + ".w1", (d, n_in), "w"), (prefix + ".b1", (d,), "b"),
                (prefix + ".w2", (n_out, d), "w"), (prefix + ".b2", (n_out,), "b")]

    if paper:
        specs = mlp("emb.trk", cfg.in_dim, d) + mlp("emb.clu", cfg.in_dim, d)
    else:
        specs = mlp("emb", cfg.in_dim, d)

    def stack(prefix, n):
        out = []
        for l in range(n):
            p = f"{prefix}.{l}."
            out += [(p + "ln1.g", (d,), "g"), (p + "ln1.b", (d,), "beta"),
                    (p + "wq", (d, d), "w"), (p + "bq", (d,), "b"),
                    (p + "wk", (d, d), "w"), (p + "bk", (d,), "b"),
                    (p + "wv", (d, d), "w"), (p + "bv", (d,), "b"),
                    (p + "wo", (d, d), "w"), (p + "bo", (d,), "b"),
                    (p + "ln2.g", (d,), "g"), (p + "ln2.b", (d,), "beta"),
                    (p + "ffn.w1", (f, d), "w"), (p + "ffn.b1", (f,), "b"),
                    (p + "ffn.w2", (d, f), "w"), (p + "ffn.b2", (d,), "b")]
        out += [(prefix + ".lnf.g", (d,), "g"), (prefix + ".lnf.b", (d,), "beta")]
        return out

    specs += stack("pid", cfg.l_pid)
    if not paper:
        specs += mlp("remb", cfg.in_dim + d, d)
    specs += stack("reg", cfg.l_reg)
    if paper:
        specs += mlp("head.bin", d, 1) + mlp("head.pid", d, cfg.n_cls - 1)
    else:
        specs += mlp("head.cls", d, cfg.n_cls)
    for name, k in REG_HEADS:
        specs += mlp(f"head.{name}", d, k)
    return specs


def make_weights(cfg: ModelConfig, seed: int, perturbed: bool = False,
                 cls_scale: float = 1.0):
    """Seeded weights: dict name -> float32 array.

    Matrices: Xavier-uniform, W ~ U(-a, a) with a = sqrt(6/(fan_in+fan_out)).
    Default: biases 0, LN gain 1, LN shift 0.  perturbed=True draws biases and
    LN shifts from U(-0.1, 0.1) and gains from 1 + U(-0.1, 0.1), so that every
    bias and normalisation parameter is exercised by parity tests.
    cls_scale multiplies the last class-head layer (weights and bias).
    """
    w = {}
    for t, (name, shape, kind) in enumerate(tensor_specs(cfg)):
        n = int(np.prod(shape))
        u = uniform(seed, STREAM_WEIGHT, t, np.arange(n, dtype=np.uint64))
        if kind == "w":
            a = math.sqrt(6.0 / (shape[0] + shape[1]))
            v = (2.0 * u - 1.0) * a
        elif kind == "g":
            v = 1.0 + (0.2 * u - 0.1 if perturbed else 0.0 * u)
        else:
            v = (0.2 * u - 0.1) if perturbed else 0.0 * u
        w[name] = v.reshape(shape).astype(np.float32)
    if cls_scale != 1.0:
        last = ("head.pid",) if cfg.arch == ARCH_PAPER else ("head.cls",)
        for h in last:
            w[h + ".w2"] = (w[h + ".w2"] * np.float32(cls_scale)).astype(np.float32)
            w[h + ".b2"] = (w[h + ".b2"] * np.float32(cls_scale)).astype(np.float32)
    return w


# --------------------------------------------------------------------------
# weight blob (read by mlpf_load_weights)
# --------------------------------------------------------------------------

BLOB_MAGIC = b"MLPF"
BLOB_VERSION = 1
NAME_BYTES = 48


def pack_blob(cfg: ModelConfig, weights) -> bytes:
    """Serialise weights into the library's blob format.

    Layout (little endian):
      char magic[4] = "MLPF"; int32 version;
      int32 in_dim, d, heads, ffn, l_pid, l_reg, n_cls, n_reg, act,
            [version 2 only: arch,] n_tensors;
      n_tensors records: char name[48]; int32 ndim; int32 shape[2];
                         float32 data[prod(shape)]
    Version 1 (arch 0 implied) is written for ARCH_SEQ, version 2 otherwise.
    """
    specs = tensor_specs(cfg)
    hdr = [cfg.in_dim, cfg.d, cfg.heads, cfg.ffn, cfg.l_pid, cfg.l_reg, cfg.n_cls, cfg.n_reg,
           cfg.act]
    version = BLOB_VERSION if cfg.arch == ARCH_SEQ else 2
    if version == 2:
        hdr.append(cfg.arch)
    hdr.append(len(specs))
    out = [BLOB_MAGIC, struct.pack("<i", version), struct.pack(f"<{len(hdr)}i", *hdr)]
    for name, shape, _ in specs:
        a = np.ascontiguousarray(weights[name], dtype=np.float32)
        assert a.shape == tuple(shape), (name, a.shape, shape)
        nb = name.encode()
        assert len(nb) < NAME_BYTES
        dims = list(shape) + [1] * (2 - len(shape))
        out.append(nb + b"\0" * (NAME_BYTES - len(nb)))
        out.append(struct.pack("<3i", len(shape), dims[0], dims[1]))
        out.append(a.tobytes())
    return b"".join(out)


def unpack_blob(blob: bytes):
    """The (ModelConfig, {tensor name: float32 array}) of a blob in the layout that
    pack_blob writes and the library's trainer exports (version 1 or 2)."""
    if blob[:4] != BLOB_MAGIC:
        raise ValueError("not a weight blob")
    (version,) = struct.unpack_from("<i", blob, 4)
    if version not in (1, 2):
        raise ValueError(f"blob version {version}")
    nh = 10 + (1 if version == 2 else 0)
    hdr = struct.unpack_from(f"<{nh}i", blob, 8)
    in_dim, d, heads, ffn, l_pid, l_reg, n_cls, n_reg, act = hdr[:9]
    arch = hdr[9] if version == 2 else ARCH_SEQ
    n_tensors = hdr[-1]
    cfg = ModelConfig(d=d, heads=heads, ffn=ffn, l_pid=l_pid, l_reg=l_reg, act=act, in_dim=in_dim,
                      n_cls=n_cls, n_reg=n_reg, arch=arch)
    off = 8 + 4 * nh
    weights = {}
    for _ in range(n_tensors):
        name = blob[off:off + NAME_BYTES].split(b"\0", 1)[0].decode()
        ndim, d0, d1 = struct.unpack_from("<3i", blob, off + NAME_BYTES)
        off += NAME_BYTES + 12
        count = d0 * d1
        a = np.frombuffer(blob, dtype="<f4", count=count, offset=off).astype(np.float32)
        weights[name] = a.reshape((d0,) if ndim == 1 else (d0, d1))
        off += 4 * count
    if off != len(blob):
        raise ValueError("trailing bytes in the blob")
    return cfg, weights


# --------------------------------------------------------------------------
# synthetic targets (supervised training without the CMS samples)
# --------------------------------------------------------------------------

STREAM_TARGET = 4
# P(target class | element type): rows = types (track, ECAL, HCAL, HF-EM, HF-HAD,
# GSF track, brem, supercluster), columns = classes (none, ch. hadron, n. hadron,
# photon, electron, muon).  Chosen so that the class is learnable from the type.
TARGET_CLASS_PROBS = np.array([
    [0.15, 0.70, 0.00, 0.00, 0.10, 0.05],
    [0.40, 0.00, 0.00, 0.60, 0.00, 0.00],
    [0.40, 0.00, 0.60, 0.00, 0.00, 0.00],
    [0.50, 0.00, 0.00, 0.50, 0.00, 0.00],
    [0.50, 0.00, 0.50, 0.00, 0.00, 0.00],
    [0.30, 0.00, 0.00, 0.00, 0.70, 0.00],
    [0.50, 0.00, 0.00, 0.50, 0.00, 0.00],
    [0.40, 0.00, 0.00, 0.60, 0.00, 0.00]])


def gen_targets(seed: int, x, cu_seqlens, first_event: int = 0):
    """Synthetic per-element targets for the supervised loss: cls [T] int32 (0 = no
    target particle, 1..5 PID class) drawn from TARGET_CLASS_PROBS by element type,
    and reg [T, 5] float32 (pT, eta, sin phi, cos phi, E): the element's own values
    perturbed by N(0, 0.3) in log pT and log E and N(0, 0.05) in eta and phi.
    Element i of event e depends only on (seed, first_event + e, i)."""
    x = np.asarray(x, np.float32)
    cu = np.asarray(cu_seqlens, np.int64)
    sizes = np.diff(cu)
    total = int(cu[-1])
    ev = np.repeat(np.arange(len(sizes), dtype=np.uint64) + np.uint64(first_event), sizes)
    idx = (np.arange(total, dtype=np.int64) - np.repeat(cu[:-1], sizes)).astype(np.uint64)
    def u(slot):
        return uniform(seed, STREAM_TARGET, ev, idx, np.uint64(slot))
    def n(slot):
        return normal(seed, STREAM_TARGET, ev, idx, np.uint64(slot))
    cls = np.zeros(total, np.int32)
    reg = np.zeros((total, 5), np.float32)
    if total == 0:
        return cls, reg
    typ = np.argmax(x[:, :N_TYPES], axis=1)
    cdf = np.cumsum(TARGET_CLASS_PROBS[typ], axis=1)
    cls[:] = np.minimum((u(0)[:, None] > cdf).sum(axis=1), N_CLS - 1)
    phi = np.arctan2(x[:, 11], x[:, 12]) + 0.05 * n(3)
    reg[:, 0] = np.exp(x[:, 8] + 0.3 * n(1))
    reg[:, 1] = x[:, 10] + 0.05 * n(2)
    reg[:, 2] = np.sin(phi)
    reg[:, 3] = np.cos(phi)
    reg[:, 4] = np.exp(x[:, 9] + 0.3 * n(4))
    return cls, reg


# deterministic truth (a learnable task for training the full model as a teacher)
TRUTH_MUON_CUT = 1.5     # first track feature above which a track is a muon
TRUTH_CLUSTER_CUT = 0.5  # a cluster makes a particle if log E > its event's mean - this


def gen_pf_truth(x, cu_seqlens):
    """Deterministic per-element truth of a PF-like rule, for training the full model
    on a learnable task (the CMS training targets are not available): cls [T] int32 and
    decoded regression targets reg [T, 5] float32 (pT, eta, sin phi, cos phi, E).

    Classes by element type: track -> muon (5) if its first track feature x[13] >
    TRUTH_MUON_CUT (a muon-system match), else charged hadron (1); GSF track -> electron
    (4); brem -> none (0); ECAL cluster -> photon (3) if its log E exceeds the mean log E
    of the event's ECAL clusters by more than -TRUTH_CLUSTER_CUT, else none (below the
    event's calibrated noise level); HCAL cluster -> neutral hadron (2) under the same
    rule over the event's HCAL clusters; HF-EM -> photon; HF-HAD -> neutral hadron;
    supercluster -> photon.  The cluster rule needs the event (a mean over other
    elements), the rest the element alone.
    Regression: tracks, GSF tracks and brems carry pT = the element's pT and
    E = pT cosh(eta) (massless); clusters carry E = the element's E and
    pT = E / cosh(eta); eta and phi are the element's own.
    """
    x = np.asarray(x, np.float64)
    cu = np.asarray(cu_seqlens, np.int64)
    sizes = np.diff(cu)
    total = int(cu[-1])
    cls = np.zeros(total, np.int32)
    reg = np.zeros((total, 5), np.float32)
    if total == 0:
        return cls, reg
    ev = np.repeat(np.arange(len(sizes)), sizes)
    typ = np.argmax(x[:, :N_TYPES], axis=1)
    loge = x[:, 9]
    cls[typ == 0] = np.where(x[typ == 0, 13] > TRUTH_MUON_CUT, 5, 1)
    cls[typ == 5] = 4
    cls[typ == 6] = 0
    for t, k in ((1, 3), (2, 2)):
        sel = typ == t
        cnt = np.bincount(ev[sel], minlength=len(sizes))
        tot = np.bincount(ev[sel], weights=loge[sel], minlength=len(sizes))
        mean = tot / np.maximum(cnt, 1)
        cls[sel] = np.where(loge[sel] > mean[ev[sel]] - TRUTH_CLUSTER_CUT, k, 0)
    cls[typ == 3] = 3
    cls[typ == 4] = 2
    cls[typ == 7] = 3
    eta = x[:, 10]
    ch = np.cosh(eta)
    is_trk = np.isin(typ, (0, 5, 6))
    pt = np.where(is_trk, np.exp(x[:, 8]), np.exp(loge) / ch)
    e = np.where(is_trk, np.exp(x[:, 8]) * ch, np.exp(loge))
    reg[:, 0] = pt
    reg[:, 1] = eta
    reg[:, 2] = x[:, 11]
    reg[:, 3] = x[:, 12]
    reg[:, 4] = e
    return cls, reg


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def workload(name: str):
    """(model config, weight seed, input seed, sizes) of a named workload."""
    if name == "event256":          # one event of 256 elements, FP32 parity
        return SMALL, 0, 101, np.array([256])
    if name == "full16":            # 16 events U{1000..6000}, full-size model
        return FULL, 1, 102, sizes_uniform(102, 16)
    if name == "prec64":            # 64 events U{1000..6000}, small model
        return SMALL, 0, 103, sizes_uniform(103, 64)
    if name == "batch512":          # 512 events LogNormal(2500, 0.5) in [100, 12000]
        return SMALL, 0, 104, sizes_lognormal(104, 512)
    if name == "paper8":            # 8 events U{1000..6000}, the architecture as printed
        return PAPER, 4, 105, sizes_uniform(105, 8)
    raise KeyError(name)
