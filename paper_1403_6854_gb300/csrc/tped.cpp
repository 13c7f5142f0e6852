// TPED haplotype reader (host code): one line per marker -- chromosome, marker
// id, genetic position (map units), physical position, then the n phased
// alleles of the sample coded 0 / 1 (Section 1.1 coding), separated by white
// space.  Markers must come in file order; the scans check that positions and
// map do not decrease.  The alleles are bit-packed while reading, straight
// into the scans' row layout (row k at rows + k * ld, haplotype h = bit h % 64
// of word h / 64, pad bits 0).
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/selscan.h"

namespace {

struct Reader {
    FILE *f = nullptr;
    char *buf = nullptr;
    size_t cap = 0;
    ~Reader()
    {
        if (f) fclose(f);
        free(buf);
    }
    // next line without the newline; false at end of file
    bool line(size_t *len)
    {
        ssize_t r = getline(&buf, &cap, f);
        if (r < 0) return false;
        while (r > 0 && (buf[r - 1] == '\n' || buf[r - 1] == '\r')) --r;
        buf[r] = 0;
        *len = (size_t)r;
        return true;
    }
};

inline const char *skip_ws(const char *p)
{
    while (*p == ' ' || *p == '\t') ++p;
    return p;
}

inline const char *field_end(const char *p)
{
    while (*p && *p != ' ' && *p != '\t') ++p;
    return p;
}

// parses one marker line; with row == NULL only counts the alleles
bool parse_line(const char *p, int32_t *count, uint64_t *row, int64_t ld, int64_t *pos,
                double *gmap)
{
    p = skip_ws(p);
    if (!*p) return false;
    p = skip_ws(field_end(p));                    // chromosome
    if (!*p) return false;
    p = skip_ws(field_end(p));                    // marker id
    if (!*p) return false;
    char *e = nullptr;
    const double g = strtod(p, &e);               // genetic position
    if (e == p || (*e && *e != ' ' && *e != '\t')) return false;
    p = skip_ws(e);
    const long long x = strtoll(p, &e, 10);       // physical position
    if (e == p || (*e && *e != ' ' && *e != '\t')) return false;
    p = skip_ws(e);
    if (pos) *pos = (int64_t)x;
    if (gmap) *gmap = g;
    int32_t h = 0;
    while (*p) {
        if ((p[0] != '0' && p[0] != '1') || (p[1] && p[1] != ' ' && p[1] != '\t')) return false;
        if (row) {
            if ((int64_t)(h >> 6) >= ld) return false;
            if (p[0] == '1') row[h >> 6] |= 1ull << (h & 63);
        }
        ++h;
        p = skip_ws(p + 1);
    }
    *count = h;
    return true;
}

}  // namespace

extern "C" int selscan_read_tped(const char *path, int32_t *n, int64_t *m, uint64_t *rows,
                                 int64_t ld, int64_t *pos_bp, double *gmap, int64_t *err_line)
{
    if (!path || !n || !m) return SELSCAN_ERR_INVALID_ARG;
    if (err_line) *err_line = 0;
    Reader r;
    r.f = fopen(path, "r");
    if (!r.f) return SELSCAN_ERR_INVALID_ARG;
    const bool fill = rows != nullptr;
    if (fill && (!pos_bp || !gmap || *n < 1 || *m < 1 || ld < (*n + 63) / 64))
        return SELSCAN_ERR_INVALID_ARG;
    int64_t k = 0;
    int32_t width = -1;
    size_t len = 0;
    while (r.line(&len)) {
        const char *p = skip_ws(r.buf);
        if (!*p) continue;                        // blank line
        if (fill && k >= *m) { if (err_line) *err_line = k + 1; return SELSCAN_ERR_INVALID_ARG; }
        int32_t c = 0;
        uint64_t *row = fill ? rows + k * ld : nullptr;
        if (row) memset(row, 0, (size_t)ld * 8);
        if (!parse_line(p, &c, row, ld, fill ? pos_bp + k : nullptr, fill ? gmap + k : nullptr) ||
            c < 1 || (width >= 0 && c != width) || (fill && c != *n)) {
            if (err_line) *err_line = k + 1;
            return SELSCAN_ERR_INVALID_ARG;
        }
        width = c;
        ++k;
    }
    if (k == 0) return SELSCAN_ERR_INVALID_ARG;
    if (fill && k != *m) { if (err_line) *err_line = k; return SELSCAN_ERR_INVALID_ARG; }
    *n = width;
    *m = k;
    return SELSCAN_OK;
}
