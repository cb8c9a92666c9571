// Shared-memory layout and the even-odd D sweep of one line, shared by the
// native FP64 and the mixed-precision kernels.
//
// Fluxes of one element are kept per (direction, field) in line-major order:
// direction r has lines (k, j) with position i, s has lines (k, i) with
// position j, t has lines (j, i) with position k.  For Nq > 8 and 8-byte
// values every line has 16 slots and slot(line, n) = 16 line + (n ^ (line & 15)):
// 16 consecutive lines, or 16 consecutive points of a line, cover all banks
// (one half-warp wavefront).  For Nq > 8 and 4-byte values lines have an odd
// number S of slots (Nq or Nq + 1) and slot(line, n) = S line + n; that holds
// for 4-byte values at Nq = 8 too (S = 9).  For 8-byte values at Nq = 8 an XOR
// swizzle slot(line, n) = 8 line + (n ^ h(line)), h(line) = (line & 6) |
// ((line >> 3) & 1), keeps the accesses free of bank conflicts when points
// write, lines read and write, and points read back (a half-warp wavefront:
// the 16 lanes need distinct (line & 1, n ^ h) pairs).
//
// The sweep uses the centro-antisymmetry of the GLL D, D[N-i][N-n] = -D[i][n]:
// with E_m = F_m + F_{N-m} and O_m = F_m - F_{N-m} (m < Nq/2),
//   S_i = a_i + b_i,  S_{N-i} = b_i - a_i,
//   a_i = sum_m De[i][m] E_m (+ D[i][c] F_c for odd Nq),  b_i = sum_m Do[i][m] O_m,
// De = (D[i][m] + D[i][N-m])/2, Do = (D[i][m] - D[i][N-m])/2, and for odd Nq the
// centre row S_c = sum_m D[c][m] O_m.  That is half the multiplies of
// S_i = sum_n D[i][n] F_n.
#pragma once

namespace numa {

// Words between consecutive lines: for 4-byte values at Nq >= 8 the smallest
// odd count >= Nq (9 at Nq = 8, 13 at Nq = 12, 17 at Nq = 16), whose odd
// stride alone keeps 32 consecutive lines on distinct banks and leaves a
// line's addresses base + n, immediate offsets without per-access arithmetic;
// 16 slots with an XOR swizzle for 8-byte values at Nq > 8; Nq otherwise.
template <int NQ, typename T>
__host__ __device__ constexpr int line_stride() {
    return (NQ >= 8 && sizeof(T) == 4) ? (NQ | 1) : (NQ > 8 ? 16 : NQ);
}

// Words of one (direction, field) block of one element: Nq^2 lines.
template <int NQ, typename T>
__host__ __device__ constexpr int block_words() {
    return NQ * NQ * line_stride<NQ, T>();
}

template <int NQ, typename T>
__device__ __forceinline__ int slot(int line, int n) {
    if constexpr (NQ >= 8 && sizeof(T) == 4)   // lines of an odd number of slots
        return line * line_stride<NQ, T>() + n;
    else if constexpr (NQ > 8)   // lines padded to 16 slots, XOR swizzle over 16
        return line * 16 + (n ^ (line & 15));
    else if constexpr (NQ == 8)
        return line * 8 + (n ^ ((line & 6) | ((line >> 3) & 1)));
    else
        return line * NQ + n;
}

// Slot of point (i, j, k) in direction d's block.  For 4-byte values at Nq = 8
// (lines of 9 slots) the r and s lines are numbered so that a warp of points
// (i = 0..7, four consecutive j, one k) touches 32 distinct banks in every
// direction: r line k + 8 j gives bank 9 k + 8 j + i, s line 4 i + (k & 3) +
// 32 (k >> 2) gives bank 4 i + j + 9 (k & 3), t line 8 j + i gives bank
// 9 i + 8 j + k (mod 32).  With the natural numbering (r line 8 k + j, s line
// 8 k + i) r and s conflict 2-way.  The sweep only needs a bijection of lines.
template <int NQ, typename T>
__device__ __forceinline__ int dir_slot(int d, int i, int j, int k) {
    if constexpr (NQ == 8 && sizeof(T) == 4) {
        if (d == 0) return slot<NQ, T>(k + 8 * j, i);
        if (d == 1) return slot<NQ, T>(4 * i + (k & 3) + 32 * (k >> 2), j);
        return slot<NQ, T>(8 * j + i, k);
    } else {
        if (d == 0) return slot<NQ, T>(NQ * k + j, i);
        if (d == 1) return slot<NQ, T>(NQ * k + i, j);
        return slot<NQ, T>(NQ * j + i, k);
    }
}

// Sweep line `line` of buf in place.  De, Do: (Nq/2)^2 row-major; Dc[r] =
// D[r][c] and Dcr[m] = D[c][m] for odd Nq.  The tables live in kernel
// parameter space, so every thread reads the same constant-bank operand.
template <int NQ, typename T, typename Tab>
__device__ __forceinline__ void sweep_line(T *buf, int line, const Tab &tab) {
    constexpr int HALF = NQ / 2;
    constexpr bool ODD = (NQ & 1) != 0;
    constexpr int C = NQ / 2;
    T F[NQ];
#pragma unroll
    for (int n = 0; n < NQ; ++n) F[n] = buf[slot<NQ, T>(line, n)];
    T E[HALF > 0 ? HALF : 1], O[HALF > 0 ? HALF : 1];
#pragma unroll
    for (int m = 0; m < HALF; ++m) {
        E[m] = F[m] + F[NQ - 1 - m];
        O[m] = F[m] - F[NQ - 1 - m];
    }
#pragma unroll
    for (int r = 0; r < HALF; ++r) {
        T a = ODD ? tab.Dc[r] * F[C] : T(0), b = T(0);
#pragma unroll
        for (int m = 0; m < HALF; ++m) {
            a = fma(tab.De[r * HALF + m], E[m], a);
            b = fma(tab.Do[r * HALF + m], O[m], b);
        }
        buf[slot<NQ, T>(line, r)] = b + a;
        buf[slot<NQ, T>(line, NQ - 1 - r)] = b - a;
    }
    if (ODD) {
        T Sc = T(0);
#pragma unroll
        for (int m = 0; m < HALF; ++m) Sc = fma(tab.Dcr[m], O[m], Sc);
        buf[slot<NQ, T>(line, C)] = Sc;
    }
}

}  // namespace numa
