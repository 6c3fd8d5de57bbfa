// Client-side format layer: CSR -> CSSC (Algorithm 5), row partitions
// (Section 4.7), chunk generation (Algorithm 2) and the totalSum rotation
// schedule (Algorithm 4).  O(nnz) host work, feeding the device layout.
#include <algorithm>
#include <numeric>

#include "internal.h"

namespace hespmv {

// Algorithm 5 on rows [r0, r1) of the CSR matrix.  Sorted row p is local row
// rm[p]; rows with equal counts keep ascending order (stable).
static void to_cssc(int32_t r0, int32_t r1, const int64_t *rowptr, const int32_t *colidx,
                    const int64_t *vals, Partition &P) {
    const int32_t rows = r1 - r0;
    P.row0 = r0;
    P.rows = rows;
    std::vector<int64_t> len(rows);
    int64_t lmax = 0;
    for (int32_t i = 0; i < rows; ++i) {
        len[i] = rowptr[r0 + i + 1] - rowptr[r0 + i];
        lmax = std::max(lmax, len[i]);
    }
    P.rm.resize(rows);
    std::iota(P.rm.begin(), P.rm.end(), 0);
    std::stable_sort(P.rm.begin(), P.rm.end(),
                     [&](int32_t a, int32_t b) { return len[a] > len[b]; });
    // number of sorted rows longer than j = height of aligned column j
    const int64_t nnz = rowptr[r1] - rowptr[r0];
    P.va.resize(nnz);
    P.src.resize(nnz);
    P.ci.resize(nnz);
    P.cp.assign(lmax + 1, 0);
    std::vector<int64_t> height(lmax, 0);
    for (int32_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < len[i]; ++j) ++height[j];
    for (int64_t j = 0; j < lmax; ++j) P.cp[j + 1] = P.cp[j] + height[j];
    // sorted row p owns entry p of every aligned column it reaches
    for (int32_t p = 0; p < rows; ++p) {
        const int32_t i = P.rm[p];
        const int64_t base = rowptr[r0 + i];
        for (int64_t j = 0; j < len[i]; ++j) {
            P.va[P.cp[j] + p] = vals ? vals[base + j] : 0;
            P.src[P.cp[j] + p] = base + j;
            P.ci[P.cp[j] + p] = colidx[base + j];
        }
    }
}

// Algorithm 2 with the padded-area capacity: a chunk of aligned columns
// [start, i) has h = height(start) rows and occupies h * (i - start) slots.
static void chunk_partition(Partition &P, int32_t part_index, int32_t s, Plan &plan) {
    const int64_t nC = (int64_t)P.cp.size() - 1;
    P.chunk0 = (int32_t)plan.chunks.size();
    int64_t i = 0;
    while (i < nC) {
        const int64_t start = i;
        const int64_t h = P.cp[start + 1] - P.cp[start];
        while (i < nC && h * (i - start + 1) <= s) ++i;
        Chunk ch;
        ch.h = (int32_t)h;
        ch.c = (int32_t)(i - start);
        ch.part = part_index;
        ch.slot0 = (int64_t)plan.slot_vals.size();
        plan.slot_vals.resize(ch.slot0 + h * ch.c, 0);
        plan.slot_ci.resize(ch.slot0 + h * ch.c, -1);
        plan.slot_src.resize(ch.slot0 + h * ch.c, -1);
        for (int32_t qc = 0; qc < ch.c; ++qc) {
            const int64_t col = start + qc;
            const int64_t n = P.cp[col + 1] - P.cp[col];
            for (int64_t p = 0; p < n; ++p) {
                plan.slot_vals[ch.slot0 + qc * h + p] = P.va[P.cp[col] + p];
                plan.slot_ci[ch.slot0 + qc * h + p] = P.ci[P.cp[col] + p];
                if (!P.src.empty()) plan.slot_src[ch.slot0 + qc * h + p] = P.src[P.cp[col] + p];
            }
        }
        plan.chunks.push_back(ch);
    }
    P.n_chunks = (int32_t)plan.chunks.size() - P.chunk0;
}

void chunk_plan(Plan &plan) {
    plan.chunks.clear();
    plan.slot_vals.clear();
    plan.slot_ci.clear();
    plan.slot_src.clear();
    for (size_t k = 0; k < plan.parts.size(); ++k) chunk_partition(plan.parts[k], (int32_t)k, plan.s, plan);
}

std::string build_plan(int32_t rows, int32_t cols, int64_t nnz, const int64_t *rowptr,
                       const int32_t *colidx, const int64_t *vals, int32_t s, Plan &plan) {
    if (rows < 0 || cols < 0 || nnz < 0 || s < 1) return "negative size";
    if (rows > 0 && !rowptr) return "rowptr is NULL";
    if (nnz > 0 && !colidx) return "colidx is NULL";
    if (rows > 0 && (rowptr[0] != 0 || rowptr[rows] != nnz)) return "rowptr[0] != 0 or rowptr[rows] != nnz";
    for (int32_t i = 0; i < rows; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return "rowptr not non-decreasing";
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] < 0 || colidx[k] >= cols) return "column index out of range";
            if (k > rowptr[i] && colidx[k] <= colidx[k - 1])
                return "column indices not strictly ascending within a row";
        }
    }
    plan = Plan();
    plan.has_values = vals != nullptr || nnz == 0;
    plan.has_src = true;
    plan.rows = rows;
    plan.cols = cols;
    plan.nnz = nnz;
    plan.s = s;
    for (int32_t r0 = 0, k = 0; r0 < rows; r0 += s, ++k) {
        Partition P;
        to_cssc(r0, std::min(rows, r0 + s), rowptr, colidx, vals, P);
        chunk_partition(P, k, s, plan);
        plan.parts.push_back(std::move(P));
    }
    return "";
}

// Halevi-Shoup totalSums over c blocks of stride r: after each doubling
// (rotate the running sum by e*r), a set bit of c adds the original
// ciphertext rotated by the new e*r.
void total_sum_steps(int32_t r, int32_t c, std::vector<int32_t> &steps,
                     std::vector<uint8_t> &from_original) {
    steps.clear();
    from_original.clear();
    if (c <= 1) return;
    int nb = 32 - __builtin_clz((unsigned)c);
    int64_t e = 1;
    for (int j = nb - 2; j >= 0; --j) {
        steps.push_back((int32_t)(e * r));
        from_original.push_back(0);
        e *= 2;
        if ((c >> j) & 1) {
            steps.push_back((int32_t)(e * r));
            from_original.push_back(1);
            e += 1;
        }
    }
}

}  // namespace hespmv
